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
__global__ void __launch_bounds__(256, (B == 16 ? 3 : 4)) ida_linear_kernel(IdaLinArgs a) {
    using Tl = Tile<B>;
    extern __shared__ __align__(16) unsigned char smem[];
    const TileSmem<B> sm(smem, 2);
    float* Ts = sm.Ts;
    float* Ys = sm.P[0];       // y, overwritten in place by z
    float* Zp = sm.P[1];       // z_prev
    uint16_t* rk = sm.rk;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start, s_end;
    __shared__ double shd[32];

    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;
    const int t = threadIdx.x;
    load_rank_table<B>(rk);
    griddep_wait();
    if (t < 32) {
        if (t == 0) s_start = a.offsets[gi0];
        if (t == 1) s_end = a.offsets[gi0 + nblk];
        tile_prefix<B>(a.counts + gi0, nblk, rel, a.status);
    }
    __syncthreads();
    const int64_t start = s_start;
    int64_t n64 = s_end - start;
    n64 = n64 < 0 ? 0 : (n64 > (int64_t)Tl::NB * B * B ? (int64_t)Tl::NB * B * B : n64);
    const int n_in = (int)n64;
    stage_in_async(Ys, a.y, start, n_in);
    if (a.z_prev) stage_in_async(Zp, a.z_prev, start, n_in);
    cp_async_commit();

    const int b = t / B, n = t % B;
    const int64_t o = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B + n) * g.Wc + (bj0 + b) * B;
    {
        float x[B];
        if (a.x && b < nblk) {
            load_f32_row<B>(a.x + o, aligned16(a.x + o), x);
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] = 0.f;
        }
        fwd_rows_to_smem<B>(x, Ts);
    }
    cp_async_wait_all();
    __syncthreads();

    // column mapping: forward DCT, residual update of the measured
    // coefficients, inverse DCT -- all in registers
    double nz = 0.0;
    {
        const int v = t % B;
        float* col = Ts + b * Tl::BLK + v;
        float x[B], c[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = col[i * Tl::LD];
        fdct<B>(x, c);
        const int sh = (int)(start & 3);
        const int r0 = rel[min(b, nblk)], m = (b < nblk) ? rel[b + 1] - r0 : 0;
        float* ys = Ys + sh + r0;
        const float* zs = Zp + sh + r0;
        const bool has_zp = a.z_prev != nullptr;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int r = rk[u * B + v];
            if (r < m) {
                const float zp = has_zp ? zs[r] : 0.f;
                const float z = (ys[r] - c[u]) + zp * a.inv_df;
                ys[r] = z;
                c[u] += z;
                nz += (double)z * (double)z;
            }
        }
        idct<B>(c, x);
#pragma unroll
        for (int i = 0; i < B; ++i) col[i * Tl::LD] = x[i];
    }
    __syncthreads();
    if (b < nblk) {
        float x[B];
        inv_rows_from_smem<B>(Ts, x);
        store_f32_row<B>(a.r + o, aligned16(a.r + o), x);
    }
    stage_out(Ys, a.z, start, n_in);
    nz = block_sum(nz, shd);
    if (t == 0)
        a.partial[(int64_t)k * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = nz;
}

template <int B>
static cudaError_t launch_lin_B(const IdaLinArgs& a, cudaStream_t s) {
    using Tl = Tile<B>;
    const size_t smem = Tl::smem_bytes(2);
    cudaError_t e = cudaFuncSetAttribute(ida_linear_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(ida_linear_kernel<B>, grid, dim3(256), smem, s, a);
}

// sigma^t = sqrt(||z^t||^2 / m) per image (Eq. 15); m = the image's
// measurement count.  Partials are summed in a fixed order.
__global__ void ida_sigma_kernel(const double* __restrict__ partial, int cpi,
                                 const int64_t* __restrict__ offsets, int64_t nB,
                                 float* __restrict__ sigma, float* __restrict__ trace, int iters,
                                 int t, uint32_t* status) {
    griddep_wait();
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
    griddep_wait();
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
            float V[8];
            fdct<8>(col, V);
#pragma unroll
            for (int u = 0; u < 8; ++u) Vs[u * 256 + t] = V[u];
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
                float c[8], qr[8];
                fdct<8>(vr, c);
#pragma unroll
                for (int v = 0; v < 8; ++v)
                    c[v] = (fabsf(c[v]) > thr || (u == 0 && v == 0)) ? c[v] : 0.f;
                idct<8>(c, qr);
#pragma unroll
                for (int j = 0; j < 8; ++j) q[u * 8 + j] = qr[j];
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
            float X[8];
            idct<8>(S, X);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) acc[kk] += X[kk];
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
    return launch_pdl(ida_sigma_kernel, dim3(g.n_img), dim3(32), 0, s, partial, ida_ctas_per_image(g), offsets,
                      (int64_t)g.n_blocks, sigma, sigma_trace, iters, t, status);
}

cudaError_t launch_tidct(const float* in, float* out, int n_img, int H, int W, const float* sigma,
                         float lambda, cudaStream_t s) {
    const size_t smem = (8 * 256 + kWin * kQS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(tidct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((W + kTW - 1) / kTW), (unsigned)((H + kTH - 1) / kTH), (unsigned)n_img);
    return launch_pdl(tidct_kernel, grid, dim3(256), smem, s, in, out, H, W, sigma, lambda);
}

}  // namespace abcs
