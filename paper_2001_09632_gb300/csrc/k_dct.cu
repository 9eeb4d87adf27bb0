// Phase-2 sensing (packed zigzag measurements, Eq. 26 rows) and the
// real-time decoder (block inverse 2D-DCT of the zero-filled measurements).
#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(dct)
}  // namespace abcs

#include "dct_tile.cuh"

namespace abcs {

namespace {

// Sum of the packed sizes of images 0 .. k-1 (warp 0 of the CTA).
ABCS_D int64_t image_base(const int64_t* img_total, int k) {
    int64_t s = 0;
    for (int j = threadIdx.x; j < k; j += 32) s += img_total[j];
    return warp_sum(s);
}

// ---------------------------------------------------------------------------
// sense_pack: C = D X D^T per block; the first m_i zigzag coefficients of
// each block are stored at coeffs[offsets[i] ...].  Offsets arrive as
// image-local exclusive prefixes (from the allocation kernel) and leave as
// global ones.  The CTA's output is one contiguous range: coalesced stores.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256) sense_pack_kernel(SenseArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    using Tl = Tile<B>;
    uint8_t* Xs = smem;
    float* Ts = reinterpret_cast<float*>(smem + Tl::XS_BYTES);
    float* Zs = Ts + Tl::TS_FLOATS;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_off0, s_base;

    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;

    if (threadIdx.x < 32) {
        const int64_t base = image_base(a.img_total, k);
        if (threadIdx.x == 0) {
            s_base = base;
            s_off0 = a.offsets[gi0];
        }
        tile_prefix<B>(a.counts + gi0, nblk, rel, nullptr);
    }
    const uint8_t* img = a.img + (int64_t)k * g.img_stride;
    load_u8_tile<B>(Xs, img, g.pitch, bi * B, bj0 * B, g.W);
    __syncthreads();
    float x[B];
#pragma unroll
    for (int n = 0; n < B; ++n) x[n] = (float)Xs[n * kTileCols + threadIdx.x];
    fwd_dct_tile_fp32<B>(x, Ts, Zs);

    const int64_t gstart = s_base + s_off0;
    if (threadIdx.x < nblk) a.offsets[gi0 + threadIdx.x] = gstart + rel[threadIdx.x];
    if (k == g.n_img - 1 && bi == g.nbh - 1 && bj0 + nblk == g.nbw && threadIdx.x == 0)
        a.offsets[(int64_t)g.n_img * g.n_blocks] = gstart + rel[nblk];
    const int total = rel[nblk];
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int b = find_block(rel, nblk, e);
        const int64_t dst = gstart + e;
        if (dst < a.capacity) a.coeffs[dst] = Zs[b * B * B + (e - rel[b])];
        else set_status(a.status, ABCS_DEV_CAPACITY);
    }
}

template <int B>
static cudaError_t launch_sense_B(const SenseArgs& a, cudaStream_t s) {
    using Tl = Tile<B>;
    const size_t smem = Tl::XS_BYTES + (Tl::TS_FLOATS + Tl::ZS_FLOATS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(sense_pack_kernel<B>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    sense_pack_kernel<B><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// reconstruct: X = D^T C D per block with C zero outside the block's first
// m_i zigzag positions.  Coefficients are gathered with coalesced loads.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256) recon_kernel(ReconArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    using Tl = Tile<B>;
    float* Ts = reinterpret_cast<float*>(smem);
    float* Zs = Ts + Tl::TS_FLOATS;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start;

    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;

    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) s_start = a.offsets[gi0];
        tile_prefix<B>(a.counts + gi0, nblk, rel, a.status);
    }
    for (int i = threadIdx.x; i < Tl::ZS_FLOATS; i += blockDim.x) Zs[i] = 0.f;
    __syncthreads();
    const int total = rel[nblk];
    const float* src = a.coeffs + s_start;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int b = find_block(rel, nblk, e);
        Zs[b * B * B + (e - rel[b])] = __ldg(src + e);
    }
    __syncthreads();
    float x[B];
    inv_dct_tile_fp32<B>(Zs, Ts, x);
    if (threadIdx.x < nblk * B) {
        const int col = bj0 * B + threadIdx.x;
        const int64_t o = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B) * g.Wc + col;
#pragma unroll
        for (int n = 0; n < B; ++n) {
            if (a.out) a.out[o + (int64_t)n * g.Wc] = x[n];
            if (a.out_u8) {
                const float v = fminf(fmaxf(rintf(x[n]), 0.f), 255.f);
                a.out_u8[o + (int64_t)n * g.Wc] = (uint8_t)v;
            }
        }
    }
}

template <int B>
static cudaError_t launch_recon_B(const ReconArgs& a, cudaStream_t s) {
    using Tl = Tile<B>;
    const size_t smem = (Tl::TS_FLOATS + Tl::ZS_FLOATS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(recon_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    recon_kernel<B><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sense_pack(const SenseArgs& a, cudaStream_t s) {
    switch (a.g.B) {
        case 4: return launch_sense_B<4>(a, s);
        case 8: return launch_sense_B<8>(a, s);
        case 16: return launch_sense_B<16>(a, s);
        case 32: return launch_sense_B<32>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reconstruct(const ReconArgs& a, cudaStream_t s) {
    switch (a.g.B) {
        case 4: return launch_recon_B<4>(a, s);
        case 8: return launch_recon_B<8>(a, s);
        case 16: return launch_recon_B<16>(a, s);
        case 32: return launch_recon_B<32>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace abcs
