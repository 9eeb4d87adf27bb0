// Phase-1 pilot estimates: block boundary variation (Eq. 19) and the DCT
// domain count n_i (Alg. 2 steps 2-4, Sec. V-B).  Both are exact integers.
#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(pilot)
}  // namespace abcs

#include "alloc_dev.cuh"
#include "dct_tile.cuh"
#include "dd_exact.cuh"

namespace abcs {

// ---------------------------------------------------------------------------
// BBV_i = sum_{j < n_S} |P(1,a+1)-P(1,a)| + |P(b+1,1)-P(b,1)|
//                     + |P(B+1,a+1)-P(B+1,a)| + |P(b+1,B+1)-P(b,B+1)|,
// a = b = X0 + jL (1-based within block i's frame).  Row B+1 / column B+1 is
// the first row / column of the block below / to the right; the bottom block
// row and the right block column use their own row B / column B instead.
// One thread per block; the per-image sum is an exact 64-bit integer.
// ---------------------------------------------------------------------------
// The loop over the n_S sample positions is unrolled four-fold so that its
// byte loads are in flight together.  With `fuse`, the last CTA of an image
// allocates it (Eqs. 22-23) and the last image allocated writes the bases.
// BBV of the blocks [c blockDim.x, (c + 1) blockDim.x) of image k; their sum
// goes to partial c of the image's ncta partials.
ABCS_D void bbv_item(const SenseArgs& a, int k, int c, int ncta, unsigned long long* sh) {
    const ImgGeom& g = a.g;
    const int64_t i = (int64_t)c * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < g.n_blocks) {
        const int B = g.B, L = a.L, X0 = a.X0, nS = a.nS;
        const int bi = (int)(i / g.nbw), bj = (int)(i - (int64_t)bi * g.nbw);
        const uint8_t* P = a.img + (int64_t)k * g.img_stride;
        const int64_t p = g.pitch;
        const int r0 = bi * B, c0 = bj * B;
        const int below = (bi + 1 < g.nbh) ? r0 + B : r0 + B - 1;
        const int right = (bj + 1 < g.nbw) ? c0 + B : c0 + B - 1;
        const uint8_t* top = P + r0 * p + c0;
        const uint8_t* bot = P + below * p + c0;
        const uint8_t* lft = P + r0 * p + c0;
        const uint8_t* rgt = P + r0 * p + right;
        int s = 0;
#pragma unroll 4
        for (int j = 0; j < nS; ++j) {
            const int a1 = X0 + j * L;   // 1-based; pair (a, a+1) -> 0-based (a-1, a)
            s += abs((int)__ldg(top + a1) - (int)__ldg(top + a1 - 1));
            s += abs((int)__ldg(lft + a1 * p) - (int)__ldg(lft + (a1 - 1) * p));
            s += abs((int)__ldg(bot + a1) - (int)__ldg(bot + a1 - 1));
            s += abs((int)__ldg(rgt + a1 * p) - (int)__ldg(rgt + (a1 - 1) * p));
        }
        a.w[(int64_t)k * g.n_blocks + i] = s;
        v = (unsigned long long)s;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0) a.wpart[(int64_t)k * ncta + c] = v;
}

__global__ void __launch_bounds__(256) bbv_kernel(SenseArgs a, int fuse) {
    __shared__ unsigned long long sh[32];
    __shared__ int64_t sh2[33];
    __shared__ int64_t sW;
    __shared__ bool s_last;
    griddep_wait();
    bbv_item(a, blockIdx.y, blockIdx.x, gridDim.x, sh);
    if (fuse) pilot_alloc_tail(a, 1, blockIdx.y, gridDim.x, sh2, &sW, &s_last);
}

// ---------------------------------------------------------------------------
// BBV pilot and allocation of one image in one CTA (1024 threads): thread t
// takes the CH or fewer consecutive blocks [t ch, t ch + ch), keeps their
// BBV_i in registers, and the CTA runs Eq. 22 (cap and redistribution of
// Sec. V-A included) and the exclusive prefix without leaving the chip.
// The last image's CTA writes the image bases.
// ---------------------------------------------------------------------------
ABCS_D int bbv_block(const SenseArgs& a, int k, int64_t i) {
    const ImgGeom& g = a.g;
    const int B = g.B, L = a.L, X0 = a.X0, nS = a.nS;
    const int ii = (int)i;                     // < n_B < 2^31
    const int bi = ii / g.nbw, bj = ii - bi * g.nbw;
    const int64_t p = g.pitch;
    const uint8_t* P = a.img + (int64_t)k * g.img_stride;
    const int r0 = bi * B, c0 = bj * B;
    const int below = (bi + 1 < g.nbh) ? r0 + B : r0 + B - 1;
    const int right = (bj + 1 < g.nbw) ? c0 + B : c0 + B - 1;
    const uint8_t* top = P + r0 * p + c0;
    const uint8_t* bot = P + below * p + c0;
    const uint8_t* rgt = P + r0 * p + right;
    // samples in predicated chunks of 8 so that all their loads are in flight together
    int s = 0;
    for (int j0 = 0; j0 < nS; j0 += 8) {
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            if (j0 + jj < nS) {
                const int a1 = X0 + (j0 + jj) * L;
                s += abs((int)__ldg(top + a1) - (int)__ldg(top + a1 - 1));
                s += abs((int)__ldg(top + a1 * p) - (int)__ldg(top + (a1 - 1) * p));
                s += abs((int)__ldg(bot + a1) - (int)__ldg(bot + a1 - 1));
                s += abs((int)__ldg(rgt + a1 * p) - (int)__ldg(rgt + (a1 - 1) * p));
            }
        }
    }
    return s;
}

// One pixel row of a block (B bytes) as 32-bit words, from a B-aligned
// address (B >= 4).
template <int B>
ABCS_D void load_row_words(const uint8_t* p, uint32_t (&w)[B / 4]) {
    if constexpr (B == 4) {
        w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
    } else if constexpr (B == 8) {
        const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        w[0] = v.x; w[1] = v.y;
    } else {
#pragma unroll
        for (int h = 0; h < B / 16; ++h) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + h);
            w[4 * h] = v.x; w[4 * h + 1] = v.y; w[4 * h + 2] = v.z; w[4 * h + 3] = v.w;
        }
    }
}

template <int NW>
ABCS_D int row_byte(const uint32_t (&w)[NW], int p) {
    uint32_t v = w[0];
#pragma unroll
    for (int q = 1; q < NW; ++q) v = (p >> 2) == q ? w[q] : v;
    return (int)((v >> (8 * (p & 3))) & 0xFFu);
}

// Eq. 19 split by the pixels each term reads: for block i with top-left
// pixel (r0, c0) and samples a = X0 + j L (j < n_S), 1-based in the block,
//   T_i = sum |P(r0, c0 + a) - P(r0, c0 + a - 1)|       (its top row)
//   L_i = sum |P(r0 + a, c0) - P(r0 + a - 1, c0)|       (its left column)
// and BBV_i = T_i + L_i + T_{block below} + L_{block to the right}, the
// block's own last row / column standing in at the image's bottom / right
// edge (EB_bj / ER_bi).  The pixel rows are read as whole B-byte vectors,
// consecutive threads taking consecutive blocks of a block row.
template <int B>
ABCS_D void bbv_terms(const SenseArgs& a, int k, int i, int16_t* sT, int16_t* sL, int16_t* sEB, int16_t* sER) {
    const ImgGeom& g = a.g;
    const int L = a.L, X0 = a.X0, nS = a.nS;
    const int bi = i / g.nbw, bj = i - bi * g.nbw;
    const int64_t p = g.pitch;
    const uint8_t* blk = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * B) * p + bj * B;
    constexpr int NW = B / 4;
    uint32_t top[NW];
    load_row_words<B>(blk, top);
    const bool last_row = bi + 1 == g.nbh, last_col = bj + 1 == g.nbw;
    int T = 0, Lc = 0, R = 0;
    // the column pairs in chunks of 4 samples, their 8 row loads in flight together
    for (int j0 = 0; j0 < nS; j0 += 4) {
        uint32_t r_lo[4][NW], r_hi[4][NW];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int a1 = X0 + min(j0 + jj, nS - 1) * L;
            load_row_words<B>(blk + (int64_t)(a1 - 1) * p, r_lo[jj]);
            load_row_words<B>(blk + (int64_t)a1 * p, r_hi[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            if (j0 + jj < nS) {
                Lc += abs((int)(r_hi[jj][0] & 0xFFu) - (int)(r_lo[jj][0] & 0xFFu));
                R += abs((int)(r_hi[jj][NW - 1] >> 24) - (int)(r_lo[jj][NW - 1] >> 24));
            }
        }
    }
    for (int j = 0; j < nS; ++j) {
        const int a1 = X0 + j * L;
        T += abs(row_byte(top, a1) - row_byte(top, a1 - 1));
    }
    sT[i] = (int16_t)T;
    sL[i] = (int16_t)Lc;
    if (last_col) sER[bi] = (int16_t)R;
    if (last_row) {
        uint32_t bot[NW];
        load_row_words<B>(blk + (int64_t)(B - 1) * p, bot);
        int Bt = 0;
        for (int j = 0; j < nS; ++j) {
            const int a1 = X0 + j * L;
            Bt += abs(row_byte(bot, a1) - row_byte(bot, a1 - 1));
        }
        sEB[bj] = (int16_t)Bt;
    }
}

template <int CH, int VB>
__global__ void __launch_bounds__(1024) bbv_image_kernel(SenseArgs a) {
    __shared__ int64_t sh[33];
    __shared__ bool s_last;
    extern __shared__ __align__(16) int16_t bbv_sm[];   // VB > 0: T, L (n_B each), EB (nbw), ER (nbh)
    griddep_wait();
    // one CTA per image leaves most SMs free: the sensing kernel may start on
    // them now and stage its first pixels (it waits for this grid before it
    // reads any count or offset)
    griddep_launch();
    const int k = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
    const int64_t nB = a.g.n_blocks;
    const int64_t ch = (nB + nt - 1) / nt;                 // <= CH (host)
    const int64_t i0 = min(nB, (int64_t)t * ch), i1 = min(nB, i0 + ch);
    int w[CH], m[CH];
    int64_t wsum = 0;
    if constexpr (VB > 0) {
        int16_t* sT = bbv_sm;
        int16_t* sL = sT + nB;
        int16_t* sEB = sL + nB;
        int16_t* sER = sEB + a.g.nbw;
        for (int i = t; i < (int)nB; i += nt) bbv_terms<VB>(a, k, i, sT, sL, sEB, sER);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = (int)(i0 + c);
            w[c] = 0;
            if (i < i1) {
                const int bi = i / a.g.nbw, bj = i - bi * a.g.nbw;
                w[c] = sT[i] + sL[i] + (bi + 1 < a.g.nbh ? sT[i + a.g.nbw] : sEB[bj]) +
                       (bj + 1 < a.g.nbw ? sL[i + 1] : sER[bi]);
            }
            wsum += w[c];
        }
    } else {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int64_t i = i0 + c;
            w[c] = (i < i1) ? bbv_block(a, k, i) : 0;
            wsum += w[c];
        }
    }
    const int64_t W = block_sum(wsum, sh);
    const int cap = a.cap;
    if (W == 0) {
#pragma unroll
        for (int c = 0; c < CH; ++c) m[c] = a.m_zz;               // L-DCT-ZZ fallback
    } else {
        // Eq. 22: m_i = floor(R BBV_i / sum BBV), capped at B^2 - 2 n_S
        int64_t E = 0;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            int64_t v = a.R * (int64_t)w[c] / W;
            if (v > cap) { E += v - cap; v = cap; }
            m[c] = (int)v;
        }
        E = block_sum(E, sh);
        // Sec. V-A: the excess goes to the blocks that are not fully measured,
        // in proportion to BBV_i, until nothing is left or nothing moves
        for (int64_t round = 0; E > 0 && round <= nB + 1; ++round) {
            int64_t wu = 0;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (m[c] < cap && w[c] > 0) wu += w[c];
            const int64_t WU = block_sum(wu, sh);
            if (WU == 0) break;
            int64_t added = 0, e2 = 0;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (m[c] < cap && w[c] > 0) {
                    const int64_t add = E * (int64_t)w[c] / WU;
                    int64_t v = m[c] + add;
                    added += add;
                    if (v > cap) { e2 += v - cap; v = cap; }
                    m[c] = (int)v;
                }
            }
            added = block_sum(added, sh);
            e2 = block_sum(e2, sh);
            if (added == 0) break;
            E = e2;
        }
    }
    int64_t local = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
        if (i0 + c < i1) local += m[c];
    int64_t total;
    int64_t run = block_exclusive_scan(local, sh, &total);
    int32_t* wk = a.w + (int64_t)k * nB;
    int32_t* ck = a.counts + (int64_t)k * nB;
    int64_t* ok = a.offsets + (int64_t)k * nB;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        if (i0 + c < i1) {
            wk[i0 + c] = w[c];
            ck[i0 + c] = m[c];
            ok[i0 + c] = run;
            run += m[c];
        }
    }
    if (t == 0) a.img_total[k] = total;
    if (a.pilot_bases) alloc_finish(a.g.n_img, a.img_total, a.img_base, a.done, sh, &s_last);
}

// Pilot CTAs per image: the number of partial sums the allocation adds up.
int pilot_ctas_per_image(const SenseArgs& a) {
    if (a.variant == ABCS_DD) {
        const int NB = kTileCols / a.g.B;
        return ((a.g.nbw + NB - 1) / NB) * a.g.nbh;
    }
    return (int)((a.g.n_blocks + 255) / 256);
}

cudaError_t launch_bbv_pilot(const SenseArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.g.n_blocks + 255) / 256), (unsigned)a.g.n_img);
    return launch_pdl(bbv_kernel, grid, dim3(256), 0, s, a, 0);
}

template <int CH, int VB>
static cudaError_t launch_bbv_image(const SenseArgs& a, cudaStream_t s) {
    const size_t smem = VB > 0 ? (size_t)(2 * a.g.n_blocks + a.g.nbw + a.g.nbh) * sizeof(int16_t) : 0;
    cudaError_t e = cudaFuncSetAttribute(bbv_image_kernel<CH, VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    return launch_pdl(bbv_image_kernel<CH, VB>, dim3((unsigned)a.g.n_img), dim3(1024), smem, s, a);
}

template <int CH>
static cudaError_t launch_bbv_image_b(const SenseArgs& a, cudaStream_t s) {
    // vector row loads need rows and images aligned to min(B, 16) bytes
    const uintptr_t al = reinterpret_cast<uintptr_t>(a.img) | (uintptr_t)a.g.pitch |
                         (uintptr_t)(a.g.n_img > 1 ? a.g.img_stride : 0);
    const uintptr_t need = (uintptr_t)(a.g.B >= 16 ? 16 : a.g.B) - 1;
    if ((al & need) == 0) {
        switch (a.g.B) {
            case 4: return launch_bbv_image<CH, 4>(a, s);
            case 8: return launch_bbv_image<CH, 8>(a, s);
            case 16: return launch_bbv_image<CH, 16>(a, s);
            case 32: return launch_bbv_image<CH, 32>(a, s);
        }
    }
    return launch_bbv_image<CH, 0>(a, s);
}

// One CTA per image when its blocks fit 16 per thread (n_B <= 16384), else
// the block-parallel pilot whose last CTA per image allocates it.
cudaError_t launch_bbv_alloc(const SenseArgs& a, cudaStream_t s) {
    const int64_t ch = (a.g.n_blocks + 1023) / 1024;
    if (ch <= 1) return launch_bbv_image_b<1>(a, s);
    if (ch <= 2) return launch_bbv_image_b<2>(a, s);
    if (ch <= 4) return launch_bbv_image_b<4>(a, s);
    if (ch <= 8) return launch_bbv_image_b<8>(a, s);
    if (ch <= 16) return launch_bbv_image_b<16>(a, s);
    dim3 grid((unsigned)((a.g.n_blocks + 255) / 256), (unsigned)a.g.n_img);
    return launch_pdl(bbv_kernel, grid, dim3(256), 0, s, a, 1);
}

// ---------------------------------------------------------------------------
// DD pilot: n_i = #{ zigzag rank j < m1 : |c_j| > T }, decided on the exact
// coefficient.  FP32 coefficients come with a rigorous error bound; any
// coefficient within that band of T is re-evaluated by the whole warp
// (dd_exact_warp): exactly in integers for (u, v) in {0, B/2}^2 (those
// coefficients are S / B with integer S), else in FP64, whose error is
// < 1e-11 here; an irrational coefficient within 1e-9 of T is flagged
// ABCS_DEV_AMBIGUOUS and counted as not exceeding.
// ---------------------------------------------------------------------------
// n_i of the blocks of tile (block row bi, tile column tx) of image k; their
// sum goes to partial `slot`.  Ts and zz are the tile's shared buffers
// (Tile<B>::FLOATS floats, B * B ranks, zz already loaded).
template <int B>
ABCS_D void dd_tile(const SenseArgs& a, int k, int bi, int tx, int64_t slot, float* Ts, const uint16_t* zz,
                    unsigned long long* sh) {
    using Tl = Tile<B>;
    const ImgGeom& g = a.g;
    const int bj0 = tx * Tl::NB;
    const int nblk = min(Tl::NB, g.nbw - bj0);
    const int t = threadIdx.x;
    const uint8_t* img = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * B) * g.pitch;
    {
        const int b = t / B, n = t % B;
        float x[B];
        if (b < nblk) {
            const uint8_t* src = img + (int64_t)n * g.pitch + (bj0 + b) * B;
            const bool vec = ((reinterpret_cast<uintptr_t>(src) & (uintptr_t)(B >= 16 ? 15 : B - 1)) == 0);
            load_u8_row<B>(src, vec, x);
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] = 0.f;
        }
        fwd_rows_to_smem<B>(x, Ts);
    }
    __syncthreads();
    fwd_cols_in_smem<B>(Ts);
    __syncthreads();

    // rigorous FP32 band: (4B + 8) u * 255 * B bounds |c_fp32 - c| for any
    // summation order of depth <= 2B (u = 2^-24)
    const float band = (4.f * B + 8.f) * 5.9604645e-8f * 255.f * B;
    const float T = (float)a.T;
    const int m1 = a.m1;
    const int w = t >> 5, lane = t & 31;
    unsigned long long mine = 0;
#pragma unroll
    for (int q = 0; q < Tl::BPW; ++q) {
        const int b = w * Tl::BPW + q;
        if (b >= nblk) break;
        const float* blk = Ts + b * Tl::BLK;
        int n = 0;
        for (int j0 = 0; j0 < m1; j0 += 32) {
            const int j = j0 + lane;
            bool hit = false, pend = false;
            if (j < m1) {
                const float c = fabsf(blk[zz[j]]);
                if (c > T + band) hit = true;
                else if (c >= T - band) pend = true;
            }
            // coefficients inside the band: decided exactly by the whole warp
            for (unsigned any = __ballot_sync(0xffffffffu, pend); any; any &= any - 1) {
                const int src = __ffs(any) - 1;
                const int p = zz_pos<B>(j0 + src);
                const bool ex = dd_exact_warp<B>(img + (bj0 + b) * B, g.pitch, p / B, p % B, a.T, a.status);
                if (lane == src) hit = ex;
            }
            n += __popc(__ballot_sync(0xffffffffu, hit));
        }
        if (lane == 0) {
            a.w[(int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0 + b] = n;
            mine += (unsigned long long)n;
        }
    }
    mine = block_sum(mine, sh);
    if (t == 0) a.wpart[slot] = mine;
}

template <int B>
__global__ void __launch_bounds__(256, 4) dd_pilot_kernel(SenseArgs a, int fuse) {
    __shared__ float Ts[Tile<B>::FLOATS];
    __shared__ uint16_t zz[B * B];
    __shared__ unsigned long long sh[32];
    __shared__ int64_t sh2[33];
    __shared__ int64_t sW;
    __shared__ bool s_last;
    load_zz_table<B>(zz);
    griddep_wait();
    const int k = blockIdx.z;
    dd_tile<B>(a, k, blockIdx.y, blockIdx.x,
               (int64_t)k * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x, Ts, zz, sh);
    if (fuse) pilot_alloc_tail(a, 2, k, gridDim.x * gridDim.y, sh2, &sW, &s_last);
}

template <int B>
static cudaError_t launch_dd_B(const SenseArgs& a, int fuse, cudaStream_t s) {
    using Tl = Tile<B>;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(dd_pilot_kernel<B>, grid, dim3(256), 0, s, a, fuse);
}

static cudaError_t launch_dd(const SenseArgs& a, int fuse, cudaStream_t s) {
    switch (a.g.B) {
        case 4: return launch_dd_B<4>(a, fuse, s);
        case 8: return launch_dd_B<8>(a, fuse, s);
        case 16: return launch_dd_B<16>(a, fuse, s);
        case 32: return launch_dd_B<32>(a, fuse, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_dd_pilot(const SenseArgs& a, cudaStream_t s) { return launch_dd(a, 0, s); }

// ---------------------------------------------------------------------------
// Uneven batch (abcs_sense_batch): one launch over the pilot work items of
// every image (BBV: 256 blocks per item; DD: one tile; L-DCT-ZZ and BBV with
// n_S = 0: one allocation-only item).  Each CTA finds its image by a binary
// search over the images' first items; the last item of an image to finish
// allocates the image (Eqs. 22-23), and the last image allocated turns the
// per-image totals into the image bases.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) pilot_batch_kernel(SenseBatchArgs b) {
    extern __shared__ __align__(16) unsigned char pb_smem[];
    __shared__ unsigned long long sh[32];
    __shared__ int64_t sh2[33];
    __shared__ int64_t sW;
    __shared__ bool s_last;
    int lo = 0, hi = b.n_img - 1;               // last image with item0 <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.imgs[mid].item0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const int k = lo;
    const SenseBatchImg& e = b.imgs[k];
    const SenseArgs a = batch_image_args(b, e, k);
    const int j = (int)blockIdx.x - e.item0;
    const int B = e.g.B;
    uint16_t* zz = reinterpret_cast<uint16_t*>(pb_smem);                  // 1024 ranks
    float* Ts = reinterpret_cast<float*>(pb_smem + 2048);
    if (e.mode == 2) {
        switch (B) {
            case 4: load_zz_table<4>(zz); break;
            case 8: load_zz_table<8>(zz); break;
            case 16: load_zz_table<16>(zz); break;
            default: load_zz_table<32>(zz); break;
        }
    }
    griddep_wait();
    bool alloc = true;
    if (e.mode == 1 || e.mode == 2) {
        if (e.mode == 1) {
            bbv_item(a, 0, j, e.cpi, sh);
        } else {
            const int ntx = (e.g.nbw + kTileCols / B - 1) / (kTileCols / B);
            const int bi = j / ntx, tx = j - bi * ntx;
            switch (B) {
                case 4: dd_tile<4>(a, 0, bi, tx, j, Ts, zz, sh); break;
                case 8: dd_tile<8>(a, 0, bi, tx, j, Ts, zz, sh); break;
                case 16: dd_tile<16>(a, 0, bi, tx, j, Ts, zz, sh); break;
                default: dd_tile<32>(a, 0, bi, tx, j, Ts, zz, sh); break;
            }
        }
        // the last of the image's items allocates it
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(a.img_done, 1u) == (unsigned)e.cpi - 1;
        }
        __syncthreads();
        alloc = s_last;
        if (alloc) {
            __threadfence();
            if (threadIdx.x == 0) *a.img_done = 0u;
        }
    } else {
        for (int64_t i = threadIdx.x; i < e.g.n_blocks; i += blockDim.x) a.w[i] = 0;   // no pilot values
    }
    if (!alloc) return;
    alloc_image(a.w, a.wpart, e.cpi, e.g.n_blocks, alloc_params(a, e.mode), 0, a.counts, a.offsets, a.img_total,
                sh2, &sW);
    alloc_finish(b.n_img, b.img_total, b.img_base, b.done, sh2, &s_last);
}

cudaError_t launch_pilot_batch(const SenseBatchArgs& b, int n_items, cudaStream_t s) {
    const size_t smem = 2048 + Tile<32>::FLOATS * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(pilot_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    return launch_pdl(pilot_batch_kernel, dim3((unsigned)n_items), dim3(256), smem, s, b);
}
cudaError_t launch_dd_alloc(const SenseArgs& a, cudaStream_t s) { return launch_dd(a, 1, s); }

}  // namespace abcs
