// Tensor-core block DCT for B = 16: sensing and reconstruction as chains of
// 16x16 matrix products on mma.sync.m16n8k16 with FP32 accumulation.
//
// One warp owns one 16x16 block at a time and keeps it in MMA fragments
// through both transform stages (the accumulator layout of the first
// product is the A-operand layout of the second), so no shared-memory
// transpose and no CTA barrier is needed.  Warps walk blocks grid-stride and
// prefetch the next block's input with cp.async while transforming the
// current one.
//
// Precisions (abcs_precision):
//   TC_FP16X2  operands split v = hi + lo in FP16; products hi*hi + lo*hi + hi*lo
//   TC_BF16X2  the same split in BF16
//   TC_BF16    single BF16 product hi*hi
// Pixels are integers <= 255, exact in FP16 and BF16, so the sensing input
// needs no split.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(tc)
}  // namespace abcs

#include "dct_tile.cuh"

namespace abcs {

namespace {

constexpr int kP16 = ABCS_TC_FP16X2, kPB16 = ABCS_TC_BF16X2, kPB1 = ABCS_TC_BF16;

template <int P>
ABCS_D uint32_t pk(float a, float b) {     // a -> low half, b -> high half
    if constexpr (P == kP16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

template <int P>
ABCS_D void unpk(uint32_t v, float& a, float& b) {
    if constexpr (P == kP16) {
        const __half2 h = *reinterpret_cast<const __half2*>(&v);
        a = __low2float(h);
        b = __high2float(h);
    } else {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&v);
        a = __low2float(h);
        b = __high2float(h);
    }
}

// (a, b) -> hi pair and lo (residual) pair
template <int P>
ABCS_D void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pk<P>(a, b);
    float ha, hb;
    unpk<P>(hi, ha, hb);
    lo = pk<P>(a - ha, b - hb);
}

template <int P>
ABCS_D void split2d(double a, double b, uint32_t& hi, uint32_t& lo) {
    hi = pk<P>((float)a, (float)b);
    float ha, hb;
    unpk<P>(hi, ha, hb);
    lo = pk<P>((float)(a - ha), (float)(b - hb));
}

template <int P>
ABCS_D void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (P == kP16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// d += A * B with both operands split (3 products) or single (1 product)
template <int P>
ABCS_D void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                      uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma<P>(d, ah, bh0, bh1);
    if constexpr (P != kPB1) {
        mma<P>(d, al, bh0, bh1);
        mma<P>(d, ah, bl0, bl1);
    }
}

// Fragment coordinates (m16n8k16, g = lane / 4, q = lane % 4):
//   A 16x16 row-major: a0 (g, 2q..2q+1), a1 (g+8, 2q..), a2 (g, 2q+8..), a3 (g+8, 2q+8..)
//   B 16x8:            b0 (2q..2q+1, g), b1 (2q+8..2q+9, g)
//   C 16x8:            c0 (g, 2q), c1 (g, 2q+1), c2 (g+8, 2q), c3 (g+8, 2q+1)
// Here k-pairs are (row k, row k+1) of B and (col k, col k+1) of A.
struct Frag {
    int g, q;
    ABCS_D Frag() : g((threadIdx.x & 31) >> 2), q(threadIdx.x & 3) {}
};

// A = M (or M^T) for the 16x16 DCT matrix M = D, from the FP64 table.
template <int P>
ABCS_D void load_a_const(bool transpose, uint32_t (&h)[4], uint32_t (&l)[4]) {
    const Frag f;
    auto e = [&](int r, int c) { return transpose ? Dd<16>(c, r) : Dd<16>(r, c); };
    split2d<P>(e(f.g, 2 * f.q), e(f.g, 2 * f.q + 1), h[0], l[0]);
    split2d<P>(e(f.g + 8, 2 * f.q), e(f.g + 8, 2 * f.q + 1), h[1], l[1]);
    split2d<P>(e(f.g, 2 * f.q + 8), e(f.g, 2 * f.q + 9), h[2], l[2]);
    split2d<P>(e(f.g + 8, 2 * f.q + 8), e(f.g + 8, 2 * f.q + 9), h[3], l[3]);
}

// B = M (or M^T), n-tiles 0 (columns 0..7) and 1 (columns 8..15).
template <int P>
ABCS_D void load_b_const(bool transpose, uint32_t (&h)[2][2], uint32_t (&l)[2][2]) {
    const Frag f;
    auto e = [&](int r, int c) { return transpose ? Dd<16>(c, r) : Dd<16>(r, c); };
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int col = f.g + 8 * nt;
        split2d<P>(e(2 * f.q, col), e(2 * f.q + 1, col), h[nt][0], l[nt][0]);
        split2d<P>(e(2 * f.q + 8, col), e(2 * f.q + 9, col), h[nt][1], l[nt][1]);
    }
}

// ---------------------------------------------------------------------------
// reconstruct: X = D^T C D.  Stage 1 Y = D^T C (A = D^T constant, B = C
// gathered from the block's zigzag-packed coefficients); stage 2 X = Y D
// (A = Y straight from stage 1's accumulators, B = D constant).
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) recon_tc_kernel(ReconArgs a, int64_t total) {
    __shared__ __align__(16) float stage[8][2][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Frag f;
    uint32_t ATh[4], ATl[4], DBh[2][2], DBl[2][2];
    load_a_const<P>(true, ATh, ATl);
    load_b_const<P>(false, DBh, DBl);
    // ranks of the 8 coefficients this lane feeds into B = C: (2q + e, g + 8 nt), e in {0,1,8,9}
    int rk[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rk[nt][i] = zz_rank(2 * f.q + (i & 1) + 8 * (i >> 1), f.g + 8 * nt, 16);

    griddep_wait();
    const ImgGeom& g = a.g;
    const int W = gridDim.x * 8;
    const int ntot = (int)total;
    int blk = blockIdx.x * 8 + warp;
    if (blk >= ntot) return;
    const unsigned nB = (unsigned)g.n_blocks, nbw = (unsigned)g.nbw;
    auto meta = [&](int b, int64_t& off, int& m) {
        off = __ldg(a.offsets + b);
        m = __ldg(a.counts + b);
        m = m < 0 ? 0 : (m > 256 ? 256 : m);
    };
    auto issue = [&](int64_t off, int m, float* dst) {
        const float* src = a.coeffs + off;
        for (int k = lane; k < m; k += 32) cp_async4(dst + k, src + k);
    };
    int64_t off0, off1 = 0;
    int m0, m1 = 0;
    meta(blk, off0, m0);
    if (blk + W < ntot) meta(blk + W, off1, m1);
    issue(off0, m0, stage[warp][0]);
    cp_async_commit();
    for (int j = 0; blk < ntot; ++j, blk += W) {
        int64_t off2 = 0;
        int m2 = 0;
        if (blk + 2 * W < ntot) meta(blk + 2 * W, off2, m2);
        if (blk + W < ntot) issue(off1, m1, stage[warp][(j + 1) & 1]);
        cp_async_commit();
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();

        const float* st = stage[warp][j & 1];
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float cv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) cv[i] = (rk[nt][i] < m0) ? st[rk[nt][i]] : 0.f;
            split2<P>(cv[0], cv[1], bh[nt][0], bl[nt][0]);
            split2<P>(cv[2], cv[3], bh[nt][1], bl[nt][1]);
        }
        float Y[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_split<P>(Y[nt], ATh, ATl, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
        uint32_t Ah[4], Al[4];
        split2<P>(Y[0][0], Y[0][1], Ah[0], Al[0]);
        split2<P>(Y[0][2], Y[0][3], Ah[1], Al[1]);
        split2<P>(Y[1][0], Y[1][1], Ah[2], Al[2]);
        split2<P>(Y[1][2], Y[1][3], Ah[3], Al[3]);
        float X[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_split<P>(X[nt], Ah, Al, DBh[nt][0], DBh[nt][1], DBl[nt][0], DBl[nt][1]);

        const unsigned k = (unsigned)blk / nB;
        const unsigned i = (unsigned)blk - k * nB;
        const unsigned bi = i / nbw, bj = i - bi * nbw;
        const int64_t o = (int64_t)k * g.Hc * g.Wc + ((int64_t)(bi * 16 + f.g) * g.Wc + bj * 16 + 2 * f.q);
        const int64_t o8 = o + 8 * (int64_t)g.Wc;
        if (a.out) {
            *reinterpret_cast<float2*>(a.out + o) = make_float2(X[0][0], X[0][1]);
            *reinterpret_cast<float2*>(a.out + o + 8) = make_float2(X[1][0], X[1][1]);
            *reinterpret_cast<float2*>(a.out + o8) = make_float2(X[0][2], X[0][3]);
            *reinterpret_cast<float2*>(a.out + o8 + 8) = make_float2(X[1][2], X[1][3]);
        }
        if (a.out_u8) {
            auto u8 = [](float v) { return (uint32_t)fminf(fmaxf(rintf(v), 0.f), 255.f); };
            *reinterpret_cast<uint16_t*>(a.out_u8 + o) = (uint16_t)(u8(X[0][0]) | (u8(X[0][1]) << 8));
            *reinterpret_cast<uint16_t*>(a.out_u8 + o + 8) = (uint16_t)(u8(X[1][0]) | (u8(X[1][1]) << 8));
            *reinterpret_cast<uint16_t*>(a.out_u8 + o8) = (uint16_t)(u8(X[0][2]) | (u8(X[0][3]) << 8));
            *reinterpret_cast<uint16_t*>(a.out_u8 + o8 + 8) = (uint16_t)(u8(X[1][2]) | (u8(X[1][3]) << 8));
        }
        __syncwarp();
        off0 = off1; m0 = m1; off1 = off2; m1 = m2;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// sense: C = D X D^T.  Stage 1 T = D X (A = D constant, B = pixels from the
// warp's staged block); stage 2 C = T D^T (A = T from the accumulators,
// B = D^T constant).  The block's first m_i zigzag coefficients are
// scattered into a per-warp staging row and copied out contiguously.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) sense_tc_kernel(SenseArgs a, int64_t total) {
    __shared__ __align__(16) uint8_t pix[8][2][256];
    __shared__ __align__(16) float ost[8][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Frag f;
    uint32_t DAh[4], DAl[4], DTh[2][2], DTl[2][2];
    load_a_const<P>(false, DAh, DAl);
    load_b_const<P>(true, DTh, DTl);
    int rk[2][4];   // ranks of this lane's accumulator positions (g + 8 (i>>1), 2q + (i&1) + 8 nt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rk[nt][i] = zz_rank(f.g + 8 * (i >> 1), 2 * f.q + (i & 1) + 8 * nt, 16);

    griddep_wait();
    const int64_t* img_base = a.img_base;
    const ImgGeom& g = a.g;
    const int W = gridDim.x * 8;
    const int ntot = (int)total;
    int blk = blockIdx.x * 8 + warp;
    if (blk >= ntot) return;
    const unsigned nB = (unsigned)g.n_blocks, nbw = (unsigned)g.nbw;
    auto issue = [&](int b, uint8_t* dst) {
        if (lane < 16) {
            const unsigned k = (unsigned)b / nB;
            const unsigned i = (unsigned)b - k * nB;
            const unsigned bi = i / nbw, bj = i - bi * nbw;
            const uint8_t* src = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * 16 + lane) * g.pitch + bj * 16;
            if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                const unsigned d = (unsigned)__cvta_generic_to_shared(dst + lane * 16);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
            } else {
                for (int c = 0; c < 16; ++c) dst[lane * 16 + c] = __ldg(src + c);
            }
        }
    };
    issue(blk, pix[warp][0]);
    cp_async_commit();
    for (int j = 0; blk < ntot; ++j, blk += W) {
        // output metadata of this block (latency hidden by the transform)
        const unsigned k = (unsigned)blk / nB;
        const int m = __ldg(a.counts + blk);
        const int64_t gstart = __ldg(img_base + k) + __ldg(a.offsets + blk);
        if (blk + W < ntot) issue(blk + W, pix[warp][(j + 1) & 1]);
        cp_async_commit();
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncwarp();

        const uint8_t* px = pix[warp][j & 1];
        uint32_t xb[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int col = f.g + 8 * nt;
            xb[nt][0] = pk<P>((float)px[(2 * f.q) * 16 + col], (float)px[(2 * f.q + 1) * 16 + col]);
            xb[nt][1] = pk<P>((float)px[(2 * f.q + 8) * 16 + col], (float)px[(2 * f.q + 9) * 16 + col]);
        }
        float T[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            mma<P>(T[nt], DAh, xb[nt][0], xb[nt][1]);
            if constexpr (P != kPB1) mma<P>(T[nt], DAl, xb[nt][0], xb[nt][1]);
        }
        uint32_t Ah[4], Al[4];
        split2<P>(T[0][0], T[0][1], Ah[0], Al[0]);
        split2<P>(T[0][2], T[0][3], Ah[1], Al[1]);
        split2<P>(T[1][0], T[1][1], Ah[2], Al[2]);
        split2<P>(T[1][2], T[1][3], Ah[3], Al[3]);
        float C[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_split<P>(C[nt], Ah, Al, DTh[nt][0], DTh[nt][1], DTl[nt][0], DTl[nt][1]);

        float* os = ost[warp];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (rk[nt][i] < m) os[rk[nt][i]] = C[nt][i];
        __syncwarp();
        if (gstart + m <= a.capacity) {
            float* dst = a.coeffs + gstart;
            for (int c = lane; c < m; c += 32) dst[c] = os[c];
        } else if (lane == 0) {
            set_status(a.status, ABCS_DEV_CAPACITY);
        }
        if (lane == 0) {
            a.offsets[blk] = gstart;
            if (blk == ntot - 1) a.offsets[ntot] = gstart + m;
        }
        __syncwarp();
    }
    cp_async_wait_all();
}

template <typename K>
cudaError_t grid_for(K kernel, int64_t total_blocks, int* grid) {
    int dev, sms, per_sm;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    if (e) return e;
    const int64_t need = (total_blocks + 7) / 8;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (int)(need < cap ? need : cap);
    return cudaSuccess;
}

template <int P>
cudaError_t launch_recon_tc_p(const ReconArgs& a, cudaStream_t s) {
    const int64_t total = (int64_t)a.g.n_img * a.g.n_blocks;
    int grid = 0;
    cudaError_t e = grid_for(recon_tc_kernel<P>, total, &grid);
    if (e) return e;
    return launch_pdl(recon_tc_kernel<P>, dim3(grid), dim3(256), 0, s, a, total);
}

template <int P>
cudaError_t launch_sense_tc_p(const SenseArgs& a, cudaStream_t s) {
    const int64_t total = (int64_t)a.g.n_img * a.g.n_blocks;
    int grid = 0;
    cudaError_t e = grid_for(sense_tc_kernel<P>, total, &grid);
    if (e) return e;
    return launch_pdl(sense_tc_kernel<P>, dim3(grid), dim3(256), 0, s, a, total);
}

}  // namespace

cudaError_t launch_recon_tc(const ReconArgs& a, cudaStream_t s) {
    if (a.g.B != 16) return cudaErrorInvalidValue;
    switch (a.precision) {
        case kP16: return launch_recon_tc_p<kP16>(a, s);
        case kPB16: return launch_recon_tc_p<kPB16>(a, s);
        case kPB1: return launch_recon_tc_p<kPB1>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sense_tc(const SenseArgs& a, cudaStream_t s) {
    if (a.g.B != 16) return cudaErrorInvalidValue;
    switch (a.precision) {
        case kP16: return launch_sense_tc_p<kP16>(a, s);
        case kPB16: return launch_sense_tc_p<kPB16>(a, s);
        case kPB1: return launch_sense_tc_p<kPB1>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace abcs
