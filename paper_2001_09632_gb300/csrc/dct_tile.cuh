// Block-row tile helpers shared by the transform kernels (internal).
//
// A CTA of 256 threads owns one block row of one image, 256 pixel columns
// wide: NB = 256 / B blocks side by side, thread t holds pixel column t
// (block t / B, in-block column t % B).  Include after ABCS_TU_TABLES(...):
// the unrolled loops read the DCT matrix through Dc<B>(k, n) with
// compile-time indices, i.e. as constant-bank operands.
#pragma once

#include "abcs_common.cuh"

namespace abcs {

template <int B>
struct Tile {
    static constexpr int NB = kTileCols / B;       // blocks per CTA
    static constexpr int TS = B + 1;               // padded row stride of Ts
    static constexpr int XS_BYTES = B * kTileCols; // uint8 pixel tile
    static constexpr int TS_FLOATS = NB * B * TS;  // stage buffer
    static constexpr int ZS_FLOATS = NB * B * B;   // zigzag-ordered coefficients
};

// Stage B rows x 256 columns of uint8 pixels into Xs[B][256] with 16-byte
// loads where the row segment is fully inside the image and aligned.
template <int B>
ABCS_D void load_u8_tile(uint8_t* Xs, const uint8_t* img, int64_t pitch, int row0, int col0,
                         int W) {
    for (int c = threadIdx.x; c < B * 16; c += blockDim.x) {
        const int r = c >> 4, ch = c & 15;
        const int col = col0 + ch * 16;
        const uint8_t* src = img + (int64_t)(row0 + r) * pitch + col;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (col + 16 <= W && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
            v = __ldg(reinterpret_cast<const uint4*>(src));
        } else if (col < W) {
            uint8_t b[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) b[i] = (col + i < W) ? __ldg(src + i) : (uint8_t)0;
            v.x = b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24);
            v.y = b[4] | (b[5] << 8) | (b[6] << 16) | ((uint32_t)b[7] << 24);
            v.z = b[8] | (b[9] << 8) | (b[10] << 16) | ((uint32_t)b[11] << 24);
            v.w = b[12] | (b[13] << 8) | (b[14] << 16) | ((uint32_t)b[15] << 24);
        }
        *reinterpret_cast<uint4*>(Xs + r * kTileCols + ch * 16) = v;
    }
}

// Forward 2D-DCT (C = D X D^T) of every block of the tile in FP32.
// In: x[n] = column t of the thread's block.  Out: Zs[blk * B*B + rank]
// in zigzag order.  Contains two __syncthreads (all threads must call).
template <int B>
ABCS_D void fwd_dct_tile_fp32(const float (&x)[B], float* Ts, float* Zs) {
    constexpr int TS = Tile<B>::TS;
    const int t = threadIdx.x;
    const int blk = t / B, m = t % B;
    // column transform: T[u][m] = sum_n D[u][n] x[n][m]
#pragma unroll
    for (int u = 0; u < B; ++u) {
        float acc = 0.f;
#pragma unroll
        for (int n = 0; n < B; ++n) acc = fmaf(Dc<B>(u, n), x[n], acc);
        Ts[(blk * B + u) * TS + m] = acc;
    }
    __syncthreads();
    // row transform: C[u][v] = sum_m T[u][m] D[v][m], thread owns row u = m
    const int u = m;
    float row[B];
#pragma unroll
    for (int j = 0; j < B; ++j) row[j] = Ts[(blk * B + u) * TS + j];
    float* zb = Zs + blk * B * B;
#pragma unroll
    for (int v = 0; v < B; ++v) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < B; ++j) acc = fmaf(row[j], Dc<B>(v, j), acc);
        zb[zz_rank(u, v, B)] = acc;
    }
    __syncthreads();
}

// Inverse 2D-DCT (X = D^T C D) of every block of the tile in FP32.
// In: Zs[blk * B*B + rank] zigzag-ordered coefficients.  Out: x[n] = column
// t of the thread's block.  Two __syncthreads.
template <int B>
ABCS_D void inv_dct_tile_fp32(const float* Zs, float* Ts, float (&x)[B]) {
    constexpr int TS = Tile<B>::TS;
    const int t = threadIdx.x;
    const int blk = t / B, m = t % B;
    const int u = m;
    const float* zb = Zs + blk * B * B;
    float crow[B];
#pragma unroll
    for (int v = 0; v < B; ++v) crow[v] = zb[zz_rank(u, v, B)];
    // row inverse: T[u][j] = sum_v C[u][v] D[v][j]
#pragma unroll
    for (int j = 0; j < B; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int v = 0; v < B; ++v) acc = fmaf(crow[v], Dc<B>(v, j), acc);
        Ts[(blk * B + u) * TS + j] = acc;
    }
    __syncthreads();
    // column inverse: X[n][m] = sum_u D[u][n] T[u][m]
    float tc[B];
#pragma unroll
    for (int k = 0; k < B; ++k) tc[k] = Ts[(blk * B + k) * TS + m];
#pragma unroll
    for (int n = 0; n < B; ++n) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < B; ++k) acc = fmaf(Dc<B>(k, n), tc[k], acc);
        x[n] = acc;
    }
    __syncthreads();
}

// Called by warp 0 only.  rel[b] = sum_{j<b} c_j for b = 0 .. nblk, with
// c_j = counts[j] clamped to [0, B*B] (a clamp sets ABCS_DEV_BADCOUNT).
// nblk <= 64: lane l owns blocks 2l and 2l+1.
template <int B>
ABCS_D void tile_prefix(const int32_t* __restrict__ counts, int nblk, int* rel, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int i0 = 2 * lane, i1 = 2 * lane + 1;
    int c0 = 0, c1 = 0;
    bool bad = false;
    if (i0 < nblk) {
        c0 = __ldg(counts + i0);
        if (c0 < 0 || c0 > B * B) { bad = true; c0 = c0 < 0 ? 0 : B * B; }
    }
    if (i1 < nblk) {
        c1 = __ldg(counts + i1);
        if (c1 < 0 || c1 > B * B) { bad = true; c1 = c1 < 0 ? 0 : B * B; }
    }
    const int pair = c0 + c1;
    int incl = pair;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - pair;
    if (i0 < nblk) rel[i0] = excl;
    if (i1 < nblk) rel[i1] = excl + c0;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) rel[nblk] = total;
    if (__any_sync(0xffffffffu, bad) && lane == 0 && status) set_status(status, ABCS_DEV_BADCOUNT);
}

// Index of the block owning packed element e, given rel[0..nb] (exclusive
// prefix of the tile's counts, rel[0] = 0): largest b with rel[b] <= e.
ABCS_D int find_block(const int* rel, int nb, int e) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rel[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace abcs
