// Phase-2 sensing (packed zigzag measurements, Eq. 26 rows) and the
// real-time decoder (block inverse 2D-DCT of the zero-filled measurements),
// FP32 CUDA-core transforms for B = 4, 8, 16, 32.
#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(dct)
}  // namespace abcs

#include "dct_tile.cuh"

namespace abcs {

namespace {

// Warp 0: tile start (image base + image-local offset) and the tile's count
// prefix.  Kept out of line: inlined, it inflates the kernel's registers.
template <int B>
__device__ __noinline__ void sense_prologue(const SenseArgs& a, int k, int64_t gi0, int nblk, int* rel,
                                            int64_t* gstart) {
    if (threadIdx.x == 0) *gstart = a.img_base[k] + a.offsets[gi0];
    tile_prefix<B>(a.counts + gi0, nblk, rel, nullptr);
}

// ---------------------------------------------------------------------------
// sense_pack: C = D X D^T per block; the first m_i zigzag coefficients of
// each block go to coeffs[offsets[i] ...].  Offsets arrive as image-local
// exclusive prefixes (from the allocation kernel) and leave as global ones.
// Row DCT (row mapping) -> smem -> column DCT (column mapping, registers) ->
// measured coefficients scattered into the tile's packed range in smem ->
// one contiguous, vectorised copy to global memory.
// ---------------------------------------------------------------------------
// One tile (block row bi, tile column tx) of image k; last_image: the tile
// writes the batch total offsets[n_img n_B] after the image's last block.
template <int B>
ABCS_D void sense_pack_tile(const SenseArgs& a, int k, int bi, int tx, bool last_image, unsigned char* smem) {
    using Tl = Tile<B>;
    const TileSmem<B> sm(smem, 1);
    float* Ts = sm.Ts;
    float* Ps = sm.P[0];
    uint16_t* rk = sm.rk;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_gstart;

    const ImgGeom& g = a.g;
    const int bj0 = tx * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;
    const int t = threadIdx.x;

    load_rank_table<B>(rk);
    griddep_wait();
    if (t < 32) sense_prologue<B>(a, k, gi0, nblk, rel, &s_gstart);
    {
        const int b = t / B, n = t % B;
        float x[B];
        if (b < nblk) {
            const uint8_t* src = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * B + n) * g.pitch +
                                 (bj0 + b) * B;
            const bool vec = ((reinterpret_cast<uintptr_t>(src) & (uintptr_t)(B >= 16 ? 15 : B - 1)) == 0);
            load_u8_row<B>(src, vec, x);
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] = 0.f;
        }
        fwd_rows_to_smem<B>(x, Ts);
    }
    __syncthreads();
    const int64_t gstart = s_gstart;
    const int sh = (int)(gstart & 3);
    {
        const int b = t / B, v = t % B;
        const float* col = Ts + b * Tl::BLK + v;
        float x[B], c[B];
#pragma unroll
        for (int n = 0; n < B; ++n) x[n] = col[n * Tl::LD];
        fdct<B>(x, c);
        if (b < nblk) {
            const int r0 = rel[b], m = rel[b + 1] - r0;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Ps + sh + r0);
#pragma unroll
            for (int u = 0; u < B; ++u) {
                const int r = rk[u * B + v];
                sts_f_lt(dst + 4u * (uint32_t)r, c[u], r, m);
            }
        }
    }
    __syncthreads();
    if (t < nblk) a.offsets[gi0 + t] = gstart + rel[t];
    if (last_image && bi == g.nbh - 1 && bj0 + nblk == g.nbw && t == 0)
        a.offsets[(int64_t)(k + 1) * g.n_blocks] = gstart + rel[nblk];
    const int total = rel[nblk];
    if (gstart + total > a.capacity) {
        if (t == 0) set_status(a.status, ABCS_DEV_CAPACITY);
        return;
    }
    stage_out(Ps, a.coeffs, gstart, total);
}

template <int B>
__global__ void __launch_bounds__(256, (B == 16 ? 3 : 4)) sense_pack_kernel(SenseArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    sense_pack_tile<B>(a, blockIdx.z, blockIdx.y, blockIdx.x, blockIdx.z == a.g.n_img - 1, smem);
}

// ---------------------------------------------------------------------------
// Uneven batch (abcs_sense_batch): one launch over the tiles of every image,
// each CTA finds its image by a binary search over the images' first tiles
// and runs the tile code of that image's block size with the image's own
// arguments (blocks, counts and offsets at the image's first block).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sense_batch_kernel(SenseBatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem[];
    int lo = 0, hi = b.n_img - 1;               // last image with tile0 <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.imgs[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const SenseBatchImg& e = b.imgs[k];
    const SenseArgs a = batch_image_args(b, e, k);
    const int NB = kTileCols / e.g.B, ntx = (e.g.nbw + NB - 1) / NB;
    const int j = (int)blockIdx.x - e.tile0, bi = j / ntx, tx = j - bi * ntx;
    const bool last = k == b.n_img - 1;
    switch (e.g.B) {
        case 4: sense_pack_tile<4>(a, 0, bi, tx, last, smem); break;
        case 8: sense_pack_tile<8>(a, 0, bi, tx, last, smem); break;
        case 16: sense_pack_tile<16>(a, 0, bi, tx, last, smem); break;
        default: sense_pack_tile<32>(a, 0, bi, tx, last, smem); break;
    }
}

// ---------------------------------------------------------------------------
// reconstruct: X = D^T C D per block with C zero outside the block's first
// m_i zigzag positions.  The tile's packed range is staged in smem with
// cp.async; the column inverse (column mapping) reads it through the rank
// table; the row inverse (row mapping) writes whole pixel rows.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256, (B == 16 ? 3 : 4)) recon_kernel(ReconArgs a) {
    using Tl = Tile<B>;
    extern __shared__ __align__(16) unsigned char smem[];
    const TileSmem<B> sm(smem, 1);
    float* Ts = sm.Ts;
    float* Ps = sm.P[0];
    uint16_t* rk = sm.rk;
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start, s_end;

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
    stage_in_async(Ps, a.coeffs, start, (int)n64);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int sh = (int)(start & 3);
    {
        const int b = t / B, v = t % B;
        float c[B], x[B];
        const int r0 = rel[min(b, nblk)], m = (b < nblk) ? rel[b + 1] - r0 : 0;
        const uint32_t src = (uint32_t)__cvta_generic_to_shared(Ps + sh + r0);
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int r = rk[u * B + v];
            c[u] = lds_f_lt(src + 4u * (uint32_t)r, r, m);
        }
        idct<B>(c, x);
        float* col = Ts + b * Tl::BLK + v;
#pragma unroll
        for (int n = 0; n < B; ++n) col[n * Tl::LD] = x[n];
    }
    __syncthreads();
    const int b = t / B, n = t % B;
    if (b < nblk) {
        float x[B];
        inv_rows_from_smem<B>(Ts, x);
        const int64_t o = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B + n) * g.Wc + (bj0 + b) * B;
        if (a.out) store_f32_row<B>(a.out + o, aligned16(a.out + o), x);
        if (a.out_u8) store_u8_row<B>(a.out_u8 + o, (reinterpret_cast<uintptr_t>(a.out_u8 + o) & 3) == 0, x);
    }
}

template <int B>
cudaError_t launch_sense_B(const SenseArgs& a, cudaStream_t s) {
    const size_t smem = Tile<B>::smem_bytes(1);
    cudaError_t e = cudaFuncSetAttribute(sense_pack_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tile<B>::NB - 1) / Tile<B>::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(sense_pack_kernel<B>, grid, dim3(256), smem, s, a);
}

template <int B>
cudaError_t launch_recon_B(const ReconArgs& a, cudaStream_t s) {
    const size_t smem = Tile<B>::smem_bytes(1);
    cudaError_t e = cudaFuncSetAttribute(recon_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tile<B>::NB - 1) / Tile<B>::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(recon_kernel<B>, grid, dim3(256), smem, s, a);
}

}  // namespace

cudaError_t launch_sense_batch(const SenseBatchArgs& b, int n_tiles, cudaStream_t s) {
    size_t smem = Tile<4>::smem_bytes(1);
    smem = Tile<8>::smem_bytes(1) > smem ? Tile<8>::smem_bytes(1) : smem;
    smem = Tile<16>::smem_bytes(1) > smem ? Tile<16>::smem_bytes(1) : smem;
    smem = Tile<32>::smem_bytes(1) > smem ? Tile<32>::smem_bytes(1) : smem;
    cudaError_t e = cudaFuncSetAttribute(sense_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    return launch_pdl(sense_batch_kernel, dim3((unsigned)n_tiles), dim3(256), smem, s, b);
}

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
