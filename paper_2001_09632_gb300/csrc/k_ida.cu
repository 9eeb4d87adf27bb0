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
// One tile: NB = 256 / B blocks of one block row.  All pointers address the
// tile's first block / pixel; coefficient indices are coeff_base +
// offsets[.].  Returns the tile's ||z||^2 (valid in thread 0).
struct LinTile {
    const int32_t* counts;
    const int64_t* offsets;
    int64_t coeff_base;
    const float* y;
    const float* x;        // NULL: x = 0
    const float* z_prev;   // NULL: z_prev = 0
    float* z;
    float* r;
    int64_t pix;           // pixel index of the tile's top-left pixel in x / r
    int Wc;                // row stride of x / r
    int nblk;
    float inv_df;
    uint32_t* status;
};

// ZP_STAGE: z_prev staged in shared memory beside y (two staging buffers);
// otherwise it is read from global memory where it is used (one buffer).
template <int B, bool ZP_STAGE = true>
ABCS_D double linear_tile(const LinTile& L, unsigned char* smem, int* rel, int64_t* s_start, double* shd) {
    using Tl = Tile<B>;
    const TileSmem<B> sm(smem, ZP_STAGE ? 2 : 1);
    float* Ts = sm.Ts;
    float* Ys = sm.P[0];       // y, overwritten in place by z
    float* Zp = sm.P[1];       // z_prev (ZP_STAGE)
    uint16_t* rk = sm.rk;
    const int t = threadIdx.x, nblk = L.nblk;
    __syncthreads();           // smem of a previous tile is free
    load_rank_table<B>(rk);
    if (t < 32) {
        if (t == 0) *s_start = L.coeff_base + L.offsets[0];
        tile_prefix<B>(L.counts, nblk, rel, L.status);
    }
    __syncthreads();
    const int64_t start = *s_start;
    const int n_in = rel[nblk];
    stage_in_async(Ys, L.y, start, n_in);
    if (ZP_STAGE && L.z_prev) stage_in_async(Zp, L.z_prev, start, n_in);
    cp_async_commit();

    const int b = t / B, n = t % B;
    const int64_t o = L.pix + (int64_t)n * L.Wc + b * B;
    {
        float x[B];
        if (L.x && b < nblk) {
            load_f32_row<B>(L.x + o, aligned16(L.x + o), x);
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
        const float* zs = ZP_STAGE ? Zp + sh + r0 : (L.z_prev ? L.z_prev + start + r0 : nullptr);
        const bool has_zp = L.z_prev != nullptr;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int r = rk[u * B + v];
            if (r < m) {
                const float zp = has_zp ? zs[r] : 0.f;
                const float z = (ys[r] - c[u]) + zp * L.inv_df;
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
        store_f32_row<B>(L.r + o, aligned16(L.r + o), x);
    }
    stage_out(Ys, L.z, start, n_in);
    return block_sum(nz, shd);
}

template <int B>
__global__ void __launch_bounds__(256, (B == 16 ? 3 : 4)) ida_linear_kernel(IdaLinArgs a) {
    using Tl = Tile<B>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start;
    __shared__ double shd[32];
    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;
    LinTile L;
    L.counts = a.counts + gi0;
    L.offsets = a.offsets + gi0;
    L.coeff_base = 0;
    L.y = a.y; L.x = a.x; L.z_prev = a.z_prev; L.z = a.z; L.r = a.r;
    L.pix = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B) * g.Wc + bj0 * B;
    L.Wc = g.Wc;
    L.nblk = min(Tl::NB, g.nbw - bj0);
    L.status = a.status;
    griddep_wait();
    L.inv_df = a.alpha ? a.alpha[k] : a.inv_df;
    const double nz = linear_tile<B>(L, smem, rel, &s_start, shd);
    if (threadIdx.x == 0)
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
// D-AMP / DAMP-D (Eqs. 24, 27): the Onsager coefficient from a Monte-Carlo
// estimate of the denoiser's divergence, div ~ b^T (D(r + eps b) - D(r)) / eps
// with eps = eps_rel max|r| per image and the caller's probe b.
// Grid (chunks, images) for the element-wise kernels.
// ---------------------------------------------------------------------------
constexpr int kDampThreads = 256;

// amax[k] = bits of max |r| over image k (non-negative floats order as
// unsigned integers); cleared by damp_clear_kernel first
__global__ void damp_clear_kernel(unsigned* __restrict__ amax) {
    griddep_wait();
    amax[blockIdx.x] = 0u;
}

__global__ void __launch_bounds__(kDampThreads) damp_amax_kernel(const float* __restrict__ r, int64_t per_img,
                                                                 unsigned* __restrict__ amax) {
    griddep_wait();
    const int k = blockIdx.y;
    const float* rk = r + (int64_t)k * per_img;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(rk[i]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax + k, __float_as_uint(m));
}

ABCS_D float damp_eps(unsigned amax_bits, float eps_rel) {
    const float e = eps_rel * __uint_as_float(amax_bits);
    return e > 0.f ? e : eps_rel;
}

__global__ void __launch_bounds__(kDampThreads) damp_perturb_kernel(const float* __restrict__ r,
                                                                    const float* __restrict__ probe, int64_t per_img,
                                                                    const unsigned* __restrict__ amax, float eps_rel,
                                                                    float* __restrict__ rp) {
    griddep_wait();
    const int k = blockIdx.y;
    const float eps = damp_eps(amax[k], eps_rel);
    const int64_t o = (int64_t)k * per_img;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        rp[o + i] = fmaf(eps, __ldg(probe + o + i), r[o + i]);
}

// per CTA: sum of b (xp - x) in FP64
__global__ void __launch_bounds__(kDampThreads) damp_div_kernel(const float* __restrict__ probe,
                                                                const float* __restrict__ xp,
                                                                const float* __restrict__ x, int64_t per_img,
                                                                double* __restrict__ partial) {
    __shared__ double sh[32];
    griddep_wait();
    const int k = blockIdx.y;
    const int64_t o = (int64_t)k * per_img;
    float a = 0.f;                                  // a thread's few terms in FP32, the CTA sum in FP64
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        a = fmaf(__ldg(probe + o + i), xp[o + i] - x[o + i], a);
    const double acc = block_sum((double)a, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = acc;
}

// one warp per image: partials in a fixed order, alpha = inv_df div / M
__global__ void damp_alpha_kernel(const double* __restrict__ partial, int chunks, const int64_t* __restrict__ offsets,
                                  int64_t nB, const unsigned* __restrict__ amax, float eps_rel, float inv_df,
                                  float* __restrict__ alpha, float* __restrict__ trace, int iters, int t,
                                  uint32_t* status) {
    griddep_wait();
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < chunks; j += 32) s += partial[(int64_t)k * chunks + j];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        const int64_t m = offsets[(int64_t)(k + 1) * nB] - offsets[(int64_t)k * nB];
        const double div = s / (double)damp_eps(amax[k], eps_rel);
        const double v = m > 0 ? (double)inv_df * div / (double)m : 0.0;
        if (!isfinite(v)) set_status(status, ABCS_DEV_NONFINITE);
        alpha[k] = (float)v;
        if (trace) trace[(int64_t)k * iters + t + 1] = (float)v;
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
constexpr int kTW = 240, kWin = kTW + 7, kCols = kTW + 14, kQS = 65;
constexpr size_t kTidctSmem = (8 * 256 + kWin * kQS) * sizeof(float);

ABCS_D int reflect(int i, int n) {
    const int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

// One 240 x TH output tile of the plain denoiser (img, dst: one image).
template <int TH>
ABCS_D void tidct_tile(const float* __restrict__ img, float* __restrict__ dst, int H, int W, int x0, int y0,
                       float thr, unsigned char* smem) {
    float* Vs = reinterpret_cast<float*>(smem);        // [8][256]
    float* Qs = Vs + 8 * 256;                          // [kWin][kQS]
    const int t = threadIdx.x;
    __syncthreads();                                   // smem of a previous tile is free

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
    const int ylast = min(y0 + TH, H);

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

template <int TH>
__global__ void __launch_bounds__(256) tidct_kernel(const float* __restrict__ in, float* __restrict__ out, int H,
                                                   int W, const float* __restrict__ sigma, float lambda) {
    extern __shared__ __align__(16) unsigned char smem[];
    griddep_wait();
    const int k = blockIdx.z;
    tidct_tile<TH>(in + (int64_t)k * H * W, out + (int64_t)k * H * W, H, W, blockIdx.x * kTW, blockIdx.y * TH,
                   lambda * __ldg(sigma + k), smem);
}

// ---------------------------------------------------------------------------
// Uneven batch: every iteration of IDA for images of different sizes and
// block sizes in ONE persistent cooperative launch.  Phases (linear step,
// per-image sigma, denoiser) are separated by grid barriers whose waits are
// bounded: a wait that exceeds `timeout` clock cycles sets
// ABCS_DEV_TIMEOUT, raises the abort flag and every CTA leaves the kernel.
// ---------------------------------------------------------------------------
#ifndef ABCS_BATCH_MINB
#define ABCS_BATCH_MINB 3
#endif

ABCS_D bool grid_sync(unsigned* bar, long long timeout, uint32_t* status, int* s_ok, bool skip_arrival = false) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile unsigned* vabort = bar + 2;
        int ok = *vabort ? 0 : 1;
        if (ok) {
            const unsigned g = *vgen;
            __threadfence();
            if (!skip_arrival && atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0u;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const long long t0 = clock64();
                while (*vgen == g) {
                    if (*vabort) { ok = 0; break; }
                    if (clock64() - t0 > timeout) {
                        atomicExch(bar + 2, 1u);
                        set_status(status, ABCS_DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// image owning tile `tile` (first-tile indices ascending)
ABCS_D int find_image(const BatchImg* imgs, int n, int tile, bool linear) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int f = linear ? __ldg(&imgs[mid].lin0) : __ldg(&imgs[mid].den0);
        if (f <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The phases of the persistent kernel are separate calls so that each is
// register-allocated on its own (inlined together they need 255 registers
// and spill, one CTA per SM).
// B = 32 reads z_prev from global memory: its shared memory (68.6 KB) then
// stays below the denoiser's, which keeps three CTAs per SM.
template <int B>
__device__ __noinline__ double linear_tile_call(const LinTile& L, unsigned char* smem, int* rel, int64_t* s_start,
                                                double* shd) {
    return linear_tile<B, (B < 32)>(L, smem, rel, s_start, shd);
}

template <int TH>
__device__ __noinline__ void tidct_tile_call(const float* img, float* dst, int H, int W, int x0, int y0, float thr,
                                             unsigned char* smem) {
    tidct_tile<TH>(img, dst, H, W, x0, y0, thr, smem);
}

template <int TH>
__global__ void __launch_bounds__(256, ABCS_BATCH_MINB) ida_batch_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int rel[kTileCols / 4 + 1];
    __shared__ int64_t s_start;
    __shared__ double shd[32];
    __shared__ int s_ok;
    const int G = gridDim.x;
    for (int t = 0; t < a.iters; ++t) {
        const float* xcur = t == 0 ? nullptr : (a.denoiser == ABCS_DEN_NONE ? ((t - 1) & 1 ? a.r1 : a.r0) : a.x);
        const float* zp = t == 0 ? nullptr : ((t - 1) & 1 ? a.z1 : a.z0);
        float* zc = (t & 1) ? a.z1 : a.z0;
        float* rc = (t & 1) ? a.r1 : a.r0;
        // linear step (Eqs. 25, 28) over every block row tile of every image
        for (int tile = blockIdx.x; tile < a.n_lin; tile += G) {
            const int k = find_image(a.imgs, a.n_img, tile, true);
            const BatchImg im = a.imgs[k];
            const int NB = kTileCols / im.B, tpr = (im.nbw + NB - 1) / NB;
            const int local = tile - im.lin0, bi = local / tpr, bj0 = (local - bi * tpr) * NB;
            const int64_t gi0 = im.blk0 + (int64_t)bi * im.nbw + bj0;
            LinTile L;
            L.counts = a.counts + gi0;
            L.offsets = a.offsets + gi0;
            L.coeff_base = im.coeff_base;
            L.y = a.y; L.x = xcur; L.z_prev = zp; L.z = zc; L.r = rc;
            L.pix = im.pix0 + (int64_t)(bi * im.B) * im.Wc + bj0 * im.B;
            L.Wc = im.Wc;
            L.nblk = min(NB, im.nbw - bj0);
            L.inv_df = a.inv_df;
            L.status = a.status;
            double nz = 0.0;
            switch (im.B) {
                case 4: nz = linear_tile_call<4>(L, smem, rel, &s_start, shd); break;
                case 8: nz = linear_tile_call<8>(L, smem, rel, &s_start, shd); break;
                case 16: nz = linear_tile_call<16>(L, smem, rel, &s_start, shd); break;
                default: nz = linear_tile_call<32>(L, smem, rel, &s_start, shd); break;
            }
            if (threadIdx.x == 0) a.partial[tile] = nz;
        }
        if (!grid_sync(a.bar, a.timeout, a.status, &s_ok, t == 0 && (int)blockIdx.x == a.skip_cta)) return;
        // sigma^t per image (Eq. 15), partials in a fixed order
        for (int k = blockIdx.x; k < a.n_img; k += G) {
            if (threadIdx.x < 32) {
                const BatchImg im = a.imgs[k];
                const int l1 = k + 1 < a.n_img ? a.imgs[k + 1].lin0 : a.n_lin;
                double s = 0.0;
                for (int j = im.lin0 + threadIdx.x; j < l1; j += 32) s += a.partial[j];
                s = warp_sum(s);
                if (threadIdx.x == 0) {
                    const int64_t last = im.blk0 + (int64_t)im.nbh * im.nbw - 1;
                    const int64_t m = a.offsets[last] + a.counts[last] - a.offsets[im.blk0];
                    const double v = m > 0 ? sqrt(s / (double)m) : 0.0;
                    if (!isfinite(v)) set_status(a.status, ABCS_DEV_NONFINITE);
                    a.sigma[k] = (float)v;
                    if (a.trace) a.trace[(int64_t)k * a.iters + t] = (float)v;
                }
            }
        }
        if (!grid_sync(a.bar, a.timeout, a.status, &s_ok)) return;
        if (a.denoiser == ABCS_DEN_TIDCT) {
            for (int tile = blockIdx.x; tile < a.n_den; tile += G) {
                const int k = find_image(a.imgs, a.n_img, tile, false);
                const BatchImg im = a.imgs[k];
                const int tx = (im.Wc + kTW - 1) / kTW;
                const int local = tile - im.den0;
                tidct_tile_call<TH>(rc + im.pix0, a.x + im.pix0, im.Hc, im.Wc, (local % tx) * kTW, (local / tx) * TH,
                                    a.lambda * a.sigma[k], smem);
            }
            if (!grid_sync(a.bar, a.timeout, a.status, &s_ok)) return;
        }
    }
}

// d[k][y][x] = m_i / B^2 of the block holding pixel (y, x) of image k; one
// image row per CTA step, B a power of two
__global__ void __launch_bounds__(256) density_kernel(ImgGeom g, const int32_t* __restrict__ counts,
                                                      float* __restrict__ out) {
    griddep_wait();
    const int rows = g.n_img * g.Hc, lb = __ffs(g.B) - 1;
    const float inv = 1.f / (float)(g.B * g.B);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = row / g.Hc, y = row - k * g.Hc;
        const int32_t* ck = counts + (int64_t)k * g.n_blocks + (int64_t)(y >> lb) * g.nbw;
        float* o = out + (int64_t)row * g.Wc;
        for (int x = threadIdx.x; x < g.Wc; x += blockDim.x) o[x] = (float)__ldg(ck + (x >> lb)) * inv;
    }
}

}  // namespace

cudaError_t launch_density(const ImgGeom& g, const int32_t* counts, float* out, cudaStream_t s) {
    const int rows = g.n_img * g.Hc;
    const unsigned grid = (unsigned)(rows < 152 * 8 ? rows : 152 * 8);
    return launch_pdl(density_kernel, dim3(grid > 0 ? grid : 1), dim3(256), 0, s, g, counts, out);
}

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

int damp_chunks(const ImgGeom& g) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const int64_t want = (152 * 8 + g.n_img - 1) / g.n_img, cap = (per_img + 4 * kDampThreads - 1) / (4 * kDampThreads);
    return (int)(want < cap ? (want > 0 ? want : 1) : (cap > 0 ? cap : 1));
}

cudaError_t launch_damp_perturb(const ImgGeom& g, const float* r, const float* probe, float eps_rel,
                                unsigned* amax, float* rp, cudaStream_t s) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const dim3 grid((unsigned)damp_chunks(g), (unsigned)g.n_img);
    cudaError_t e = launch_pdl(damp_clear_kernel, dim3((unsigned)g.n_img), dim3(1), 0, s, amax);
    if (!e) e = launch_pdl(damp_amax_kernel, grid, dim3(kDampThreads), 0, s, r, per_img, amax);
    if (!e)
        e = launch_pdl(damp_perturb_kernel, grid, dim3(kDampThreads), 0, s, r, probe, per_img, (const unsigned*)amax,
                       eps_rel, rp);
    return e;
}

cudaError_t launch_damp_alpha(const ImgGeom& g, const int64_t* offsets, const float* probe, const float* xp,
                              const float* x, const unsigned* amax, float eps_rel, float inv_df, double* partial,
                              float* alpha, float* alpha_trace, int iters, int t, uint32_t* status, cudaStream_t s) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const int chunks = damp_chunks(g);
    cudaError_t e = launch_pdl(damp_div_kernel, dim3((unsigned)chunks, (unsigned)g.n_img), dim3(kDampThreads), 0, s,
                               probe, xp, x, per_img, partial);
    if (!e)
        e = launch_pdl(damp_alpha_kernel, dim3((unsigned)g.n_img), dim3(32), 0, s, (const double*)partial, chunks,
                       offsets, (int64_t)g.n_blocks, amax, eps_rel, inv_df, alpha, alpha_trace, iters, t, status);
    return e;
}

size_t ida_batch_smem(unsigned used_b_mask) {
    size_t s = kTidctSmem;
    if (used_b_mask & 4) s = s > Tile<4>::smem_bytes(2) ? s : Tile<4>::smem_bytes(2);
    if (used_b_mask & 8) s = s > Tile<8>::smem_bytes(2) ? s : Tile<8>::smem_bytes(2);
    if (used_b_mask & 16) s = s > Tile<16>::smem_bytes(2) ? s : Tile<16>::smem_bytes(2);
    if (used_b_mask & 32) s = s > Tile<32>::smem_bytes(1) ? s : Tile<32>::smem_bytes(1);
    return s;
}

int ida_batch_tile_w() { return kTW; }

template <int TH>
static cudaError_t launch_batch_th(const BatchArgs& a, int ctas_per_sm, size_t smem, cudaStream_t s, int* grid_out) {
    cudaError_t e = cudaFuncSetAttribute(ida_batch_kernel<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int dev, sms, per_sm;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ida_batch_kernel<TH>, 256, smem))) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int use = ctas_per_sm < per_sm ? ctas_per_sm : per_sm;
    int grid = sms * use;
    const int work = a.n_lin > a.n_den ? a.n_lin : a.n_den;
    if (grid > work) grid = work > 0 ? work : 1;
    if (grid_out) *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ida_batch_kernel<TH>, a);
}

// th: denoiser tile height (32 or 64); ctas_per_sm: requested residency
cudaError_t launch_ida_batch(const BatchArgs& a, int th, int ctas_per_sm, size_t smem, cudaStream_t s, int* grid) {
    if (th == 32) return launch_batch_th<32>(a, ctas_per_sm, smem, s, grid);
    return launch_batch_th<64>(a, ctas_per_sm, smem, s, grid);
}

cudaError_t launch_tidct(const float* in, float* out, int n_img, int H, int W, const float* sigma,
                         float lambda, cudaStream_t s) {
    constexpr int TH = 64;
    const size_t smem = kTidctSmem;
    cudaError_t e = cudaFuncSetAttribute(tidct_kernel<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((W + kTW - 1) / kTW), (unsigned)((H + TH - 1) / TH), (unsigned)n_img);
    return launch_pdl(tidct_kernel<TH>, grid, dim3(256), smem, s, in, out, H, W, sigma, lambda);
}

}  // namespace abcs
