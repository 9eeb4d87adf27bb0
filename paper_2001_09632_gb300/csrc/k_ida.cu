// IDA (Sec. VI): the linear part of one iteration (Eqs. 25, 28 and the
// residual norm of Eq. 15) and the plain denoiser D_sigma.
#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(ida)
}  // namespace abcs

#include "dct_tile.cuh"

namespace abcs {

namespace {

// ---------------------------------------------------------------------------
// Linear step, fused per block:  c = DCT(x);  for the measured ranks
//   z = y - c + z_prev / D_F           (Eq. 25 + Onsager term alpha = 1/D_F, Eq. 28)
//   c <- c + z                          (adds A^T z in the DCT domain)
// then r = IDCT(c) = x + A^T z, and the CTA's share of ||z||^2 in FP64.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256) ida_linear_kernel(IdaLinArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    using Tl = Tile<B>;
    float* Ts = reinterpret_cast<float*>(smem);
    float* Zs = Ts + Tl::TS_FLOATS;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start;
    __shared__ double shd[32];

    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) s_start = a.offsets[gi0];
        tile_prefix<B>(a.counts + gi0, nblk, rel, a.status);
    }

    const bool valid = threadIdx.x < nblk * B;
    const int64_t o = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B) * g.Wc + bj0 * B + threadIdx.x;
    float x[B];
#pragma unroll
    for (int n = 0; n < B; ++n) x[n] = (a.x && valid) ? __ldg(a.x + o + (int64_t)n * g.Wc) : 0.f;
    fwd_dct_tile_fp32<B>(x, Ts, Zs);

    double nz = 0.0;
    const int total = rel[nblk];
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int b = find_block(rel, nblk, e);
        const int r = e - rel[b];
        const int64_t gi = s_start + e;
        float* zc = Zs + b * B * B + r;
        const float c = *zc;
        const float zp = a.z_prev ? __ldg(a.z_prev + gi) : 0.f;
        const float z = (__ldg(a.y + gi) - c) + zp * a.inv_df;
        a.z[gi] = z;
        *zc = c + z;
        nz += (double)z * (double)z;
    }
    __syncthreads();
    inv_dct_tile_fp32<B>(Zs, Ts, x);
    if (valid) {
#pragma unroll
        for (int n = 0; n < B; ++n) a.r[o + (int64_t)n * g.Wc] = x[n];
    }
    nz = block_sum(nz, shd);
    if (threadIdx.x == 0)
        a.partial[(int64_t)k * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = nz;
}

template <int B>
static cudaError_t launch_lin_B(const IdaLinArgs& a, cudaStream_t s) {
    using Tl = Tile<B>;
    const size_t smem = (Tl::TS_FLOATS + Tl::ZS_FLOATS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(ida_linear_kernel<B>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    ida_linear_kernel<B><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

// sigma^t = sqrt(||z^t||^2 / m) per image (Eq. 15); m = the image's
// measurement count.  Partials are summed in a fixed order.
__global__ void ida_sigma_kernel(const double* __restrict__ partial, int cpi,
                                 const int64_t* __restrict__ offsets, int64_t nB,
                                 float* __restrict__ sigma, float* __restrict__ trace, int iters,
                                 int t, uint32_t* status) {
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < cpi; j += 32) s += partial[(int64_t)k * cpi + j];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        const int64_t m = offsets[(int64_t)(k + 1) * nB] - offsets[(int64_t)k * nB];
        const double v = m > 0 ? sqrt(s / (double)m) : 0.0;
        if (!isfinite(v)) set_status(status, ABCS_DEV_NONFINITE);
        sigma[k] = (float)v;
        if (trace) trace[(int64_t)k * iters + t] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// Plain denoiser: translation-invariant 8x8 DCT hard thresholding.  Every
// pixel is the mean, over the 64 8x8 windows that contain it, of the window
// after an orthonormal DCT, zeroing of the AC coefficients with
// |c| <= lambda sigma, and the inverse DCT.  Outside the image the input is
// extended half-sample symmetrically.
//
// A CTA produces a 240 x 64 output tile.  It walks the window rows wy from
// y0-7 to y0+63; per window row:
//   (a) column DCT of 8 input rows, shared by all windows of the row
//       (thread per input column, sliding 8-row register window);
//   (b) thread per window: row DCT, threshold, row inverse -> Q (smem);
//   (c) thread per output column: overlap-add of the 8 windows covering it
//       and the column inverse, accumulated in 8 sliding registers; the top
//       row is complete and written out.
// Every output accumulates in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kTW = 240, kTH = 64, kWin = kTW + 7, kCols = kTW + 14, kQS = 65;

ABCS_D int reflect(int i, int n) {
    const int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

__global__ void __launch_bounds__(256) tidct_kernel(const float* __restrict__ in,
                                                   float* __restrict__ out, int H, int W,
                                                   const float* __restrict__ sigma, float lambda) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* Vs = reinterpret_cast<float*>(smem);        // [8][256]
    float* Qs = Vs + 8 * 256;                          // [kWin][kQS]
    const int k = blockIdx.z;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    const float* img = in + (int64_t)k * H * W;
    float* dst = out + (int64_t)k * H * W;
    const float thr = lambda * __ldg(sigma + k);
    const int t = threadIdx.x;

    // (a) state: this thread's input column and its 8-row window
    const bool has_col = t < kCols;
    const int xc = reflect(x0 - 7 + t, W);
    float col[8];
    if (has_col) {
#pragma unroll
        for (int i = 0; i < 8; ++i) col[i] = __ldg(img + (int64_t)reflect(y0 - 7 + i, H) * W + xc);
    }
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
    const int ylast = min(y0 + kTH, H);

    for (int wy = y0 - 7; wy < ylast; ++wy) {
        if (has_col) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float v = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) v = fmaf(Dc<8>(u, i), col[i], v);
                Vs[u * 256 + t] = v;
            }
#pragma unroll
            for (int i = 0; i < 7; ++i) col[i] = col[i + 1];
            if (wy + 8 < ylast + 7) col[7] = __ldg(img + (int64_t)reflect(wy + 8, H) * W + xc);
        }
        __syncthreads();
        if (t < kWin) {
            float* q = Qs + t * kQS;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float vr[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) vr[j] = Vs[u * 256 + t + j];
                float c[8];
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    float s = 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) s = fmaf(vr[j], Dc<8>(v, j), s);
                    c[v] = (fabsf(s) > thr || (u == 0 && v == 0)) ? s : 0.f;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float s = 0.f;
#pragma unroll
                    for (int v = 0; v < 8; ++v) s = fmaf(c[v], Dc<8>(v, j), s);
                    q[u * 8 + j] = s;
                }
            }
        }
        __syncthreads();
        if (t < kTW) {
            float S[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                float s = 0.f;
#pragma unroll
                for (int d = 0; d < 8; ++d) s += Qs[(t + d) * kQS + u * 8 + (7 - d)];
                S[u] = s;
            }
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                float s = acc[kk];
#pragma unroll
                for (int u = 0; u < 8; ++u) s = fmaf(Dc<8>(u, kk), S[u], s);
                acc[kk] = s;
            }
            if (wy >= y0 && x0 + t < W) dst[(int64_t)wy * W + x0 + t] = acc[0] * (1.f / 64.f);
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) acc[kk] = acc[kk + 1];
            acc[7] = 0.f;
        }
    }
}

}  // namespace

int ida_ctas_per_image(const ImgGeom& g) {
    const int NB = kTileCols / g.B;
    return ((g.nbw + NB - 1) / NB) * g.nbh;
}

cudaError_t launch_ida_linear(const IdaLinArgs& a, cudaStream_t s) {
    switch (a.g.B) {
        case 4: return launch_lin_B<4>(a, s);
        case 8: return launch_lin_B<8>(a, s);
        case 16: return launch_lin_B<16>(a, s);
        case 32: return launch_lin_B<32>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_ida_sigma(const ImgGeom& g, const int64_t* offsets, const double* partial,
                             float* sigma, float* sigma_trace, int iters, int t, uint32_t* status,
                             cudaStream_t s) {
    ida_sigma_kernel<<<g.n_img, 32, 0, s>>>(partial, ida_ctas_per_image(g), offsets, g.n_blocks,
                                            sigma, sigma_trace, iters, t, status);
    return cudaGetLastError();
}

cudaError_t launch_tidct(const float* in, float* out, int n_img, int H, int W, const float* sigma,
                         float lambda, cudaStream_t s) {
    const size_t smem = (8 * 256 + kWin * kQS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(tidct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((W + kTW - 1) / kTW), (unsigned)((H + kTH - 1) / kTH), (unsigned)n_img);
    tidct_kernel<<<grid, 256, smem, s>>>(in, out, H, W, sigma, lambda);
    return cudaGetLastError();
}

}  // namespace abcs
