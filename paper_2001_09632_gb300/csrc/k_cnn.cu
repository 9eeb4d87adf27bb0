// Learned residual denoiser for IDA (a DnCNN-style network, Sec. VI-4):
//   conv3x3 4->32 + ReLU, 6 x [conv3x3 32->32 + ReLU], conv3x3 32->1,
//   x_hat = r - 255 * net(r / 255, sigma / 255, d, tau), zero 'same' padding,
//   d = the measured fraction m_i / B^2 of the pixel's block (or 0),
//   tau = the iteration input (min(t, 8) / 8 in IDA iteration t).
// Activations and mid-layer weights are BF16 (activations chunk-planar:
// four planes of 8 channels per image); every sum accumulates in FP32.  All
// layers are implicit GEMMs on the tensor cores: the forward 32->32 layers
// and the last (32 -> 1, weights split BF16 hi + lo) on tcgen05 (bulk-copy
// fed, TMEM accumulators, 128-pixel rows, operands read from shared memory by
// descriptor), the input-gradient 32->32 layers on mma.sync (persistent
// CTAs, weights resident, double-buffered tiles fed with ldmatrix), the
// first layer (4 channels: r / 255, sigma / 255, d, tau) in FP16 mma.sync.
//
// Training (fwd + bwd + Adam) reuses the same conv kernel for the input
// gradient (weights transposed in (ci, co) and flipped in the tap, epilogue
// = ReLU mask of the layer below); weight gradients are accumulated per CTA
// in FP32 and reduced in a fixed order (deterministic).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "abcs_common.cuh"
#include "umma.cuh"

namespace abcs {

// ---------------------------------------------------------------------------
// Parameter layout (FP32, the same as the FP64 oracle's):
//   for l in 0..7: w_l[co][ci][3][3], then b_l[co]
// channel plan: (4->32), 6 x (32->32), (32->1).
// ---------------------------------------------------------------------------
constexpr int kC = 32, kMid = 6, kIn = 4;
constexpr int kW0 = kC * kIn * 9, kB0 = kC;
constexpr int kWm = kC * kC * 9, kBm = kC;
constexpr int kW7 = kC * 9, kB7 = 1;
constexpr int kParams = kW0 + kB0 + kMid * (kWm + kBm) + kW7 + kB7;   // 56,961

ABCS_HD int param_off_w(int l) {
    return l == 0 ? 0 : (l <= kMid ? kW0 + kB0 + (l - 1) * (kWm + kBm) : kW0 + kB0 + kMid * (kWm + kBm));
}
ABCS_HD int param_off_b(int l) {
    return param_off_w(l) + (l == 0 ? kW0 : (l <= kMid ? kWm : kW7));
}

// Packed device weights (one buffer, offsets in bytes).
struct CnnPacked {
    float w0[kC][kIn][9];           // first layer, FP32 [co][ci][tap]
    float b0[kC];
    __nv_bfloat16 wc[kMid][9][kC][kC];   // mid layers, forward [tap][co][ci]
    __nv_bfloat16 wd[kMid][9][kC][kC];   // mid layers, input-gradient [tap'][ci][co], tap' = 8 - tap
    float bm[kMid][kC];
    float w7[kC][9];                // last layer, FP32 [ci][tap]
    float b7;
    alignas(16) __nv_bfloat16 w7t[9][16][kC];   // last layer for the tensor cores: [tap][col][ci], col 0 = BF16 hi, 1 = lo
};

namespace {

constexpr int TH = 8, TW = 32, IH = TH + 2, IW = TW + 2;

// Activations and their gradients are stored chunk-planar, [n][4][H][W][8]:
// image k, 16-byte chunk c / 8 (channels 8 (c / 8) .. 8 (c / 8) + 7), row y,
// pixel x, channel c % 8.  A row of one chunk is contiguous, so tile loads
// and stores move whole lines.
ABCS_D int64_t act_off(int k, int y, int x, int c, int H, int W) {
    return ((((int64_t)k * 4 + (c >> 3)) * H + y) * W + x) * 8 + (c & 7);
}

// four 8 x 8 BF16 matrices from a shared-window address
ABCS_D void ldmatrix_x4s(uint32_t (&r)[4], uint32_t a) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

ABCS_D void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

ABCS_D uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// (max(a, 0), max(b, 0)) rounded to BF16 and packed, a in the low half
ABCS_D uint32_t pack_bf16_relu(float a, float b) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(b), "f"(a));
    return d;
}


// ---------------------------------------------------------------------------
// 32 -> 32 conv3x3 as an implicit GEMM (M = pixels, N = 32, K = 9 x 32).
// EPI 0: out = ReLU(acc + bias)            (forward)
// EPI 1: out = acc * [mask > 0]            (input gradient through a ReLU)
// Persistent CTAs: the layer's weights are loaded once, the input tiles
// (8 x 32 outputs, 10 x 34 inputs with a zero halo) are double-buffered with
// cp.async (zero fill outside the image), so the next tile streams in while
// the tensor cores work on the current one.  A pixel's 32 channels take 64
// bytes of shared memory; the 16-byte chunks are XOR-swizzled by
// (pixel >> 1) & 3, which keeps every ldmatrix conflict-free.
// ---------------------------------------------------------------------------
ABCS_D int swz(int p, int c) { return p * 32 + ((c ^ ((p >> 1) & 3)) << 3); }   // bf16 index

ABCS_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
ABCS_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

ABCS_D void cp_async16_zfill(void* sdst, const void* gsrc, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    const int nbytes = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(nbytes) : "memory");
}

// The staged input tile keeps a row stride of IWP = 40 pixels (34 used):
// since IWP / 2 is a multiple of 4, moving by whole rows (and by 16 pixels)
// leaves the swizzle term unchanged, so every ldmatrix address of the inner
// loop is one of eight per-lane bases plus a compile-time offset.
constexpr int IWP = 40;
constexpr int kTileElems = IH * IWP * kC;         // bf16 of one staged input tile
constexpr int kWElems = 9 * kC * kC;              // bf16 of one layer's weights
constexpr size_t kConvSmem = (size_t)(2 * kTileElems + kWElems) * 2;

template <int EPI>
__global__ void __launch_bounds__(256, 3) conv32_kernel(const __nv_bfloat16* __restrict__ in, int n, int H,
                                                        int W, const __nv_bfloat16* __restrict__ wts,
                                                        const float* __restrict__ bias,
                                                        const __nv_bfloat16* __restrict__ mask,
                                                        __nv_bfloat16* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* tw = reinterpret_cast<__nv_bfloat16*>(smem);        // [9 * 32 rows (tap, co)][32 ci]
    __nv_bfloat16* tb0 = tw + kWElems;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH, per_img = tx * ty;
    const int ntiles = per_img * n;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    for (int c = t; c < 9 * kC * 4; c += 256)        // weights do not depend on the previous kernel
        cp_async16_zfill(tw + swz(c >> 2, c & 3), wts + (c >> 2) * kC + (c & 3) * 8, true);
    griddep_wait();
    auto origin = [&](int tl, int& k, int& x0, int& y0) {
        k = tl / per_img;
        const int rem = tl - k * per_img, by = rem / tx;
        x0 = (rem - by * tx) * TW;
        y0 = by * TH;
    };
    auto stage = [&](int tl, __nv_bfloat16* dst) {
        int k, x0, y0;
        origin(tl, k, x0, y0);
        for (int c = t; c < IH * IW * 4; c += 256) {
            const int ch = c / (IH * IW), px = c - ch * (IH * IW);
            const int py = px / IW, pxx = px - py * IW;
            const int yy = y0 - 1 + py, xx = x0 - 1 + pxx;
            const bool v = yy >= 0 && yy < H && xx >= 0 && xx < W;
            cp_async16_zfill(dst + swz(py * IWP + pxx, ch), v ? in + act_off(k, yy, xx, 8 * ch, H, W) : in, v);
        }
    };
    stage(tile, tb0);
    cp_async_commit();
    const int G = gridDim.x;
    const int arow = lane & 15, achk = lane >> 4;                                // A: pixel row, chunk
    const int brow = (lane & 7) + (lane >> 4) * 8, bchk = (lane >> 3) & 1;      // B: co row, chunk
    const int g = lane >> 2, q = lane & 3;
    // per-lane byte offsets: A for tap column dx and k-step ks (row warp, dy = 0), B for ks (tap 0)
    uint32_t aoff[3][2], boff[2];
#pragma unroll
    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) aoff[dx][ks] = 2u * (uint32_t)swz(warp * IWP + dx + arow, 2 * ks + achk);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) boff[ks] = 2u * (uint32_t)swz(brow, 2 * ks + bchk);
    const uint32_t tw_s = (uint32_t)__cvta_generic_to_shared(tw);
    for (int i = 0; tile < ntiles; ++i, tile += G) {
        __nv_bfloat16* cur = tb0 + (i & 1) * kTileElems;
        if (tile + G < ntiles) stage(tile + G, tb0 + ((i + 1) & 1) * kTileElems);
        cp_async_commit();
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();

        float acc[2][4][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int nn = 0; nn < 4; ++nn)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[h][nn][e] = 0.f;
        const uint32_t cur_s = (uint32_t)__cvta_generic_to_shared(cur);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t a0[4], a1[4], b01[4], b23[4];
                const uint32_t aa = cur_s + aoff[dx][ks] + 2u * (uint32_t)(dy * IWP * kC);
                const uint32_t bb = tw_s + boff[ks] + 2u * (uint32_t)(tap * kC * kC);
                ldmatrix_x4s(a0, aa);
                ldmatrix_x4s(a1, aa + 2u * 16 * kC);
                ldmatrix_x4s(b01, bb);
                ldmatrix_x4s(b23, bb + 2u * 16 * kC);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t(&a)[4] = h ? a1 : a0;
                    mma_bf16(acc[h][0], a, b01[0], b01[1]);
                    mma_bf16(acc[h][1], a, b01[2], b01[3]);
                    mma_bf16(acc[h][2], a, b23[0], b23[1]);
                    mma_bf16(acc[h][3], a, b23[2], b23[3]);
                }
            }
        }
        __syncthreads();                     // every warp is done reading `cur`
        // epilogue through `cur`: [TH * TW pixels][32 channels], then 16-byte stores
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int nn = 0; nn < 4; ++nn) {
                const int co = nn * 8 + 2 * q;
                const float b0 = (EPI == 0) ? __ldg(bias + co) : 0.f, b1 = (EPI == 0) ? __ldg(bias + co + 1) : 0.f;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int px = warp * TW + h * 16 + g + 8 * half;
                    float v0 = acc[h][nn][2 * half] + b0, v1 = acc[h][nn][2 * half + 1] + b1;
                    if (EPI == 0) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
                    *reinterpret_cast<uint32_t*>(cur + swz(px, nn) + 2 * q) = pack_bf16(v0, v1);
                }
            }
        __syncthreads();
        int k, x0, y0;
        origin(tile, k, x0, y0);
        for (int c = t; c < TH * TW * 4; c += 256) {
            const int ch = c / (TH * TW), px = c - ch * (TH * TW);
            const int yy = y0 + px / TW, xx = x0 + px % TW;
            if (yy >= H || xx >= W) continue;
            uint4 v = *reinterpret_cast<const uint4*>(cur + swz(px, ch));
            const int64_t o = act_off(k, yy, xx, 8 * ch, H, W);
            if (EPI == 1) {
                const uint4 m = __ldg(reinterpret_cast<const uint4*>(mask + o));
                const uint32_t* mw = reinterpret_cast<const uint32_t*>(&m);
                uint32_t* vw = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    // a BF16 activation is > 0 iff its sign bit is clear and it is not +0
                    const uint32_t lo = (mw[e] & 0xFFFFu), hi = (mw[e] >> 16);
                    const uint32_t keep_lo = (lo != 0 && !(lo & 0x8000u)) ? 0xFFFFu : 0u;
                    const uint32_t keep_hi = (hi != 0 && !(hi & 0x8000u)) ? 0xFFFF0000u : 0u;
                    vw[e] &= keep_lo | keep_hi;
                }
            }
            *reinterpret_cast<uint4*>(out + o) = v;
        }
        __syncthreads();                     // `cur` is staged into again two tiles later
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// First layer on the tensor cores: an implicit GEMM with K = (tap, channel),
// k = 4 tap + ci over the channels (r / 255, sigma / 255, d, 0), 36 values
// zero-padded to 48, FP16 operands, FP32 accumulation.  Each shared pixel
// holds the two pairs (r / 255, sigma / 255) and (d, 0) as FP16x2 words
// (zero outside the image: the zero padding of every channel), so one
// 32-bit shared load is one A-fragment register.  Persistent CTAs keep the
// weight fragments in registers, prefetch the next tile's inputs during
// the current tile's MMAs, and store straight from the accumulators.
// ---------------------------------------------------------------------------
ABCS_D void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

ABCS_D uint32_t pack_f16(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// weight pair p = 2 tap + half of output channel co: (w[r], w[sigma]) or (w[d], w[tau])
ABCS_D uint32_t w0_pair(const CnnPacked* P, int co, int p) {
    if (p >= 18) return 0u;
    const int tap = p >> 1;
    return (p & 1) ? pack_f16(__ldg(&P->w0[co][2][tap]), __ldg(&P->w0[co][3][tap]))
                   : pack_f16(__ldg(&P->w0[co][0][tap]), __ldg(&P->w0[co][1][tap]));
}

// the iteration input of image k: tau[k], or tau0 for every image
ABCS_D float tau_of(const float* tau, float tau0, int k) { return tau ? __ldg(tau + k) : tau0; }

__global__ void __launch_bounds__(256, 3) cnn_first_tc_kernel(const float* __restrict__ r,
                                                              const float* __restrict__ sigma,
                                                              const float* __restrict__ dens,
                                                              const float* __restrict__ tau, float tau0, int n,
                                                              int H, int W, const CnnPacked* __restrict__ P,
                                                              __nv_bfloat16* __restrict__ out) {
    __shared__ uint32_t tin[IH * IW * 2];                 // per pixel: (r, sigma), (d, tau) as FP16x2
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, g = lane >> 2, q = lane & 3;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH, per_img = tx * ty, ntiles = per_img * n;
    const int G = gridDim.x;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    // B fragments: ks covers pairs 8 ks .. 8 ks + 7; b0 = pair 8 ks + q, b1 = pair 8 ks + q + 4
    uint32_t bf[3][4][2];
    float bias[4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int ks = 0; ks < 3; ++ks) {
            bf[ks][nt][0] = w0_pair(P, 8 * nt + g, 8 * ks + q);
            bf[ks][nt][1] = w0_pair(P, 8 * nt + g, 8 * ks + q + 4);
        }
        bias[nt][0] = __ldg(&P->b0[8 * nt + 2 * q]);
        bias[nt][1] = __ldg(&P->b0[8 * nt + 2 * q + 1]);
    }
    // A fragments: pair p = 8 ks + q + 4 j (tap p / 2, half p % 2) of pixel (row, col) is
    // the shared word 2 ((row + dy) IW + col + dx) + half; pairs 18.. are the K padding
    int aoff[3][2];
#pragma unroll
    for (int ks = 0; ks < 3; ++ks)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int p = 8 * ks + q + 4 * j, tap = p >> 1;
            aoff[ks][j] = p < 18 ? 2 * ((tap / 3) * IW + tap % 3) + (p & 1) : -1;
        }
    constexpr int NPT = (IH * IW + 255) / 256;
    int fy[NPT], fx[NPT];                                 // this thread's halo pixels in a tile
#pragma unroll
    for (int e = 0; e < NPT; ++e) {
        const int c = t + 256 * e;
        fy[e] = c < IH * IW ? c / IW - 1 : -(1 << 20);    // -> outside every image when unused
        fx[e] = c % IW - 1;
    }
    const int64_t ps = (int64_t)H * W * 8;                // elements per chunk plane
    griddep_wait();
    uint32_t pre[NPT][2];
    auto origin = [&](int tl, int& k, int& y0, int& x0) {
        k = tl / per_img;
        const int rem = tl - k * per_img, by = rem / tx;
        y0 = by * TH;
        x0 = (rem - by * tx) * TW;
    };
    auto fetch = [&](int tl) {
        int k, y0, x0;
        origin(tl, k, y0, x0);
        const float s255 = __ldg(sigma + k) * (1.f / 255.f);
        const float tk = tau_of(tau, tau0, k);
        const float* rk = r + (int64_t)k * H * W;
        const float* dk = dens ? dens + (int64_t)k * H * W : nullptr;
#pragma unroll
        for (int e = 0; e < NPT; ++e) {
            const int yy = y0 + fy[e], xx = x0 + fx[e];
            const bool in_img = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const int o = yy * W + xx;
            pre[e][0] = in_img ? pack_f16(__ldg(rk + o) * (1.f / 255.f), s255) : 0u;
            pre[e][1] = in_img ? pack_f16(dk ? __ldg(dk + o) : 0.f, tk) : 0u;
        }
    };
    fetch(tile);
    for (; tile < ntiles; tile += G) {
        __syncthreads();                                  // the previous tile's reads of tin are done
#pragma unroll
        for (int e = 0; e < NPT; ++e) {
            const int c = t + 256 * e;
            if (c < IH * IW) {
                tin[2 * c] = pre[e][0];
                tin[2 * c + 1] = pre[e][1];
            }
        }
        __syncthreads();
        if (tile + G < ntiles) fetch(tile + G);           // in flight during this tile's MMAs and stores
        int k, y0, x0;
        origin(tile, k, y0, x0);
        const int y = y0 + warp;
        __nv_bfloat16* ob = out + (int64_t)k * 4 * ps + ((int64_t)y * W + x0 + g) * 8 + 2 * q;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float acc[4][4];                              // starts at the bias
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[nt][e] = bias[nt][e & 1];
            const int base = 2 * (warp * IW + 16 * h + g);
#pragma unroll
            for (int ks = 0; ks < 3; ++ks) {
                uint32_t a[4];
                a[0] = aoff[ks][0] >= 0 ? tin[base + aoff[ks][0]] : 0u;
                a[1] = aoff[ks][0] >= 0 ? tin[base + 16 + aoff[ks][0]] : 0u;
                a[2] = aoff[ks][1] >= 0 ? tin[base + aoff[ks][1]] : 0u;
                a[3] = aoff[ks][1] >= 0 ? tin[base + 16 + aoff[ks][1]] : 0u;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_f16(acc[nt], a, bf[ks][nt][0], bf[ks][nt][1]);
            }
            // bias, ReLU, BF16: lanes (g, q) of one store cover 8 pixels x 16 bytes, one full line
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int x = x0 + 16 * h + g + 8 * half;
                if (y < H && x < W) {
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        *reinterpret_cast<uint32_t*>(ob + nt * ps + (16 * h + 8 * half) * 8) =
                            pack_bf16_relu(acc[nt][2 * half], acc[nt][2 * half + 1]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Packing: FP32 parameters (oracle layout) -> CnnPacked.
// ---------------------------------------------------------------------------
__global__ void cnn_pack_kernel(const float* __restrict__ prm, CnnPacked* __restrict__ P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kW0) (&P->w0[0][0][0])[i] = prm[i];                        // [co][ci][tap] == [co][ci][3][3]
    if (i < kB0) P->b0[i] = prm[kW0 + i];
    if (i < kMid * kWm) {
        const int l = i / kWm, j = i % kWm;                              // j over [co][ci][tap]
        const int co = j / (kC * 9), ci = (j / 9) % kC, tap = j % 9;
        const __nv_bfloat16 v = __float2bfloat16_rn(prm[param_off_w(l + 1) + j]);
        P->wc[l][tap][co][ci] = v;
        P->wd[l][8 - tap][ci][co] = v;
    }
    if (i < kMid * kBm) P->bm[i / kBm][i % kBm] = prm[param_off_b(i / kBm + 1) + i % kBm];
    if (i < kW7) (&P->w7[0][0])[i] = prm[param_off_w(7) + i];              // [ci][tap] == [0][ci][3][3]
    if (i < 9 * 16 * kC) {                                                  // [tap][col][ci]
        const int tap = i / (16 * kC), col = (i / kC) % 16, ci = i % kC;
        const float w = prm[param_off_w(7) + ci * 9 + tap];
        const __nv_bfloat16 hi = __float2bfloat16_rn(w);
        const __nv_bfloat16 lo = __float2bfloat16_rn(w - __bfloat162float(hi));
        P->w7t[tap][col][ci] = col == 0 ? hi : (col == 1 ? lo : __float2bfloat16_rn(0.f));
    }
    if (i == 0) P->b7 = prm[param_off_b(7)];
}

// ---------------------------------------------------------------------------
// Training pieces.
// ---------------------------------------------------------------------------
// resid = r/255 - n - clean/255; loss += resid^2 / numel; g = -2 resid / numel
__global__ void cnn_loss_kernel(const float* __restrict__ n, const float* __restrict__ r,
                                const float* __restrict__ clean, int64_t numel, float* __restrict__ g,
                                double* __restrict__ part) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < numel; i += (int64_t)gridDim.x * blockDim.x) {
        const float res = __ldg(r + i) * (1.f / 255.f) - __ldg(n + i) - __ldg(clean + i) * (1.f / 255.f);
        g[i] = -2.f * res / (float)numel;
        s += (double)res * res;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s / (double)numel;
}

// input gradient of the last layer, times the ReLU mask of its input:
// d[q][ci] = [act[q][ci] > 0] * sum_tap w7[ci][tap] g[q - off(tap)]
__global__ void __launch_bounds__(256) cnn_last_bwd_kernel(const float* __restrict__ g, const __nv_bfloat16* __restrict__ act,
                                                           int H, int W, const CnnPacked* __restrict__ P,
                                                           __nv_bfloat16* __restrict__ d) {
    __shared__ float tg[IH * IW];
    __shared__ float sw[kC * 9];
    const int t = threadIdx.x, k = blockIdx.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const float* gi = g + (int64_t)k * H * W;
    for (int c = t; c < IH * IW; c += 256) {
        const int yy = y0 - 1 + c / IW, xx = x0 - 1 + c % IW;
        tg[c] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(gi + (int64_t)yy * W + xx) : 0.f;
    }
    for (int c = t; c < kC * 9; c += 256) sw[c] = (&P->w7[0][0])[c];
    __syncthreads();
    const int py = t / TW, px = t % TW, yy = y0 + py, xx = x0 + px;
    if (yy >= H || xx >= W) return;
    // out[p] = sum_tap w[tap] in[p + off(tap)]  =>  d_in[q] = sum_tap w[tap] g[q - off(tap)]
    float gv[9];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) gv[tap] = tg[(py + 2 - tap / 3) * IW + (px + 2 - tap % 3)];
    uint32_t res[16];
#pragma unroll
    for (int ci = 0; ci < kC; ci += 2) {
        float v[2] = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) v[e] = fmaf(sw[(ci + e) * 9 + tap], gv[tap], v[e]);
        const float2 av = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(act + act_off(k, yy, xx, ci, H, W)));
        res[ci / 2] = pack_bf16(av.x > 0.f ? v[0] : 0.f, av.y > 0.f ? v[1] : 0.f);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(d + act_off(k, yy, xx, 8 * c, H, W)) =
            make_uint4(res[4 * c], res[4 * c + 1], res[4 * c + 2], res[4 * c + 3]);
}

// Weight gradients of a 32 -> 32 layer: dW[co][ci][tap] = sum_p g[p][co] in[p + off(tap)][ci],
// db[co] = sum_p g[p][co].  Persistent CTAs over 8 x 32 tiles; each CTA
// writes its FP32 partial (kWm + kBm values) to part[blockIdx.x].
__global__ void __launch_bounds__(256) wgrad32_kernel(const __nv_bfloat16* __restrict__ in,
                                                      const __nv_bfloat16* __restrict__ g, int n, int H, int W,
                                                      float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* tin = reinterpret_cast<float*>(smem);            // [IH*IW][33]
    float* tgg = tin + IH * IW * 33;                        // [TH*TW][33]
    const int t = threadIdx.x;
    // thread t owns co = t / 8 and ci in {ci0 .. ci0 + 3} (ci0 = 4 (t % 8)), all 9 taps: 36 weights
    const int co = t >> 3, ci0 = (t & 7) * 4;
    float acc[4][9];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 9; ++b) acc[a][b] = 0.f;
    float accb = 0.f;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH, ntiles = tx * ty * n;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int k = tile / (tx * ty), rem = tile % (tx * ty);
        const int y0 = (rem / tx) * TH, x0 = (rem % tx) * TW;
        __syncthreads();
        for (int c = t; c < IH * IW * kC / 2; c += 256) {
            const int px = c / (kC / 2), cp = (c % (kC / 2)) * 2;
            const int yy = y0 - 1 + px / IW, xx = x0 - 1 + px % IW;
            float2 v = make_float2(0.f, 0.f);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(
                    in + act_off(k, yy, xx, cp, H, W)));
            tin[px * 33 + cp] = v.x;
            tin[px * 33 + cp + 1] = v.y;
        }
        for (int c = t; c < TH * TW * kC / 2; c += 256) {
            const int px = c / (kC / 2), cp = (c % (kC / 2)) * 2;
            const int yy = y0 + px / TW, xx = x0 + px % TW;
            float2 v = make_float2(0.f, 0.f);
            if (yy < H && xx < W)
                v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(
                    g + act_off(k, yy, xx, cp, H, W)));
            tgg[px * 33 + cp] = v.x;
            tgg[px * 33 + cp + 1] = v.y;
        }
        __syncthreads();
        for (int p = 0; p < TH * TW; ++p) {
            const float gv = tgg[p * 33 + co];
            accb += gv;
            const int py = p / TW, px = p % TW;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const float* ip = tin + ((py + tap / 3) * IW + px + tap % 3) * 33 + ci0;
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[a][tap] = fmaf(gv, ip[a], acc[a][tap]);
            }
        }
    }
    float* dst = part + (int64_t)blockIdx.x * (kWm + kBm);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) dst[(co * kC + ci0 + a) * 9 + tap] = acc[a][tap];
    if ((t & 7) == 0) dst[kWm + co] = accb;
}

// Weight gradients of the first layer (inputs r/255, sigma/255, d, tau; g: 32 ch).
__global__ void __launch_bounds__(256) wgrad_first_kernel(const float* __restrict__ r, const float* __restrict__ sigma,
                                                          const float* __restrict__ dens, const float* __restrict__ tau,
                                                          float tau0, const __nv_bfloat16* __restrict__ g, int n, int H,
                                                          int W, float* __restrict__ part) {
    __shared__ float tr[IH * IW];
    __shared__ float tv[IH * IW];        // 1 inside the image, 0 in the zero padding
    __shared__ float td[IH * IW];        // density, 0 in the padding
    __shared__ float tgg[TH * TW][33];
    const int t = threadIdx.x;
    // thread t: co = t / 8; thread sub = t % 8 owns (ci, tap) weights 5 sub .. 5 sub + 4 of the 36
    constexpr int kPer = 5;
    static_assert(8 * kPer >= kIn * 9, "first-layer weights per output channel");
    const int co = t >> 3, sub = t & 7;
    float acc[kPer] = {};
    float accb = 0.f;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH, ntiles = tx * ty * n;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int k = tile / (tx * ty), rem = tile % (tx * ty);
        const int y0 = (rem / tx) * TH, x0 = (rem % tx) * TW;
        const float s255 = __ldg(sigma + k) * (1.f / 255.f);
        const float tk = tau_of(tau, tau0, k);
        __syncthreads();
        for (int c = t; c < IH * IW; c += 256) {
            const int yy = y0 - 1 + c / IW, xx = x0 - 1 + c % IW;
            const bool in = yy >= 0 && yy < H && xx >= 0 && xx < W;
            const int64_t o = ((int64_t)k * H + yy) * W + xx;
            tr[c] = in ? __ldg(r + o) * (1.f / 255.f) : 0.f;
            tv[c] = in ? 1.f : 0.f;
            td[c] = (in && dens) ? __ldg(dens + o) : 0.f;
        }
        for (int c = t; c < TH * TW * kC / 2; c += 256) {
            const int px = c / (kC / 2), cp = (c % (kC / 2)) * 2;
            const int yy = y0 + px / TW, xx = x0 + px % TW;
            float2 v = make_float2(0.f, 0.f);
            if (yy < H && xx < W)
                v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(
                    g + act_off(k, yy, xx, cp, H, W)));
            tgg[px][cp] = v.x;
            tgg[px][cp + 1] = v.y;
        }
        __syncthreads();
        for (int p = 0; p < TH * TW; ++p) {
            const float gv = tgg[p][co];
            if (sub == 0) accb += gv;
            const int py = p / TW, px = p % TW;
#pragma unroll
            for (int e = 0; e < kPer; ++e) {
                const int idx = sub * kPer + e;            // 0..35 = ci * 9 + tap
                if (idx < kIn * 9) {
                    const int ci = idx / 9, tap = idx % 9;
                    const int ti = (py + tap / 3) * IW + px + tap % 3;
                    const float in = ci == 0 ? tr[ti] : (ci == 1 ? s255 * tv[ti] : (ci == 2 ? td[ti] : tk * tv[ti]));
                    acc[e] = fmaf(gv, in, acc[e]);
                }
            }
        }
    }
    float* dst = part + (int64_t)blockIdx.x * (kW0 + kB0);
#pragma unroll
    for (int e = 0; e < kPer; ++e)
        if (sub * kPer + e < kIn * 9) dst[co * kIn * 9 + sub * kPer + e] = acc[e];
    if (sub == 0) dst[kW0 + co] = accb;
}

// Weight gradients of the last layer: dW7[ci][tap] = sum_p g[p] in[p + off(tap)][ci], db7 = sum_p g[p].
__global__ void __launch_bounds__(256) wgrad_last_kernel(const __nv_bfloat16* __restrict__ in, const float* __restrict__ g,
                                                         int n, int H, int W, float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* tin = reinterpret_cast<float*>(smem);    // [IH*IW][33]
    __shared__ float tg[TH * TW];
    const int t = threadIdx.x;
    // 288 weights + 1 bias over 256 threads: thread t handles (ci, tap) pairs t and t + 256
    float acc[2] = {0.f, 0.f};
    float accb = 0.f;
    const int tx = (W + TW - 1) / TW, ty = (H + TH - 1) / TH, ntiles = tx * ty * n;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int k = tile / (tx * ty), rem = tile % (tx * ty);
        const int y0 = (rem / tx) * TH, x0 = (rem % tx) * TW;
        __syncthreads();
        for (int c = t; c < IH * IW * kC / 2; c += 256) {
            const int px = c / (kC / 2), cp = (c % (kC / 2)) * 2;
            const int yy = y0 - 1 + px / IW, xx = x0 - 1 + px % IW;
            float2 v = make_float2(0.f, 0.f);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(
                    in + act_off(k, yy, xx, cp, H, W)));
            tin[px * 33 + cp] = v.x;
            tin[px * 33 + cp + 1] = v.y;
        }
        {
            const int yy = y0 + t / TW, xx = x0 + t % TW;
            tg[t] = (yy < H && xx < W) ? __ldg(g + ((int64_t)k * H + yy) * W + xx) : 0.f;
        }
        __syncthreads();
        for (int p = 0; p < TH * TW; ++p) {
            const float gv = tg[p];
            if (t == 0) accb += gv;
            const int py = p / TW, px = p % TW;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int idx = t + 256 * e;
                if (idx < kW7) {
                    const int ci = idx / 9, tap = idx % 9;
                    acc[e] = fmaf(gv, tin[((py + tap / 3) * IW + px + tap % 3) * 33 + ci], acc[e]);
                }
            }
        }
    }
    float* dst = part + (int64_t)blockIdx.x * (kW7 + kB7);
    for (int e = 0; e < 2; ++e)
        if (t + 256 * e < kW7) dst[t + 256 * e] = acc[e];
    if (t == 0) dst[kW7] = accb;
}

// grad[off + j] = sum_c part[c][j], fixed order
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, int len, float* __restrict__ grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s += part[(int64_t)c * len + j];
    grad[j] = s;
}

__global__ void reduce_loss_kernel(const double* __restrict__ part, int n, float* __restrict__ loss) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += part[i];
    s = warp_sum(s);
    if (threadIdx.x == 0) *loss = (float)s;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int cnn_param_count() { return kParams; }
size_t cnn_packed_bytes() { return sizeof(CnnPacked); }

cudaError_t cnn_pack(const float* params, void* packed, cudaStream_t s) {
    cnn_pack_kernel<<<(kMid * kWm + 255) / 256, 256, 0, s>>>(params, static_cast<CnnPacked*>(packed));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 32 -> 32 forward layer on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators, bulk asynchronous copies).  Per input row i of 130 pixels and per dx one
// row-level implicit GEMM against the three dy taps at once:
//   D[128 px][dy, co] += A[128 px][32 ci] B[32 ci][dy, co]
// as two MMAs of K = 16 (M = 128, N up to 96), FP32 accumulation in tensor
// memory; the dy column block lands on output row i - dy's accumulator
// (rows are kept in reverse order, so those blocks are adjacent).
// A is read straight from the staged input tile: the tile is kept
// k-chunk-major (four planes of 8 channels, 16 bytes per pixel, pixels
// contiguous), so each (plane, input row) of the tile is one contiguous run
// of the chunk-planar activations (one bulk copy of up to 2080 bytes), and
// the A matrix of input row i and column shift dx is the same no-swizzle
// K-major layout starting (i * 130 + dx) pixels on.  (A tensor-map copy of
// 8-channel boxes moves 16 bytes per request; whole runs move full lines.)
//   tile: TH output rows x 128 pixels; input TH + 2 rows x 130 pixels (the
//   producer zeroes the halo outside the image); TH = 4 for the 32 -> 32
//   layers (3 input buffers), TH = 8 for the last layer (2 input buffers)
//   warp 0: producer, 4 (TH + 2) bulk copies per tile (full/empty
//           mbarriers, the full one counting the bytes)
//   warp 1: tensor-memory allocation and the MMA issuer (2 accumulator
//           buffers of TH rows x NC columns)
//   warps 2-9: epilogue; warp w reads TMEM lanes 32 (w % 4) of rows
//           (w - 2) / 4 + 2 m (tcgen05.ld), adds the bias,
//           applies the ReLU, converts to BF16; each store of a warp
//           covers 32 consecutive pixels of one plane (512 bytes)
// Every mbarrier wait is bounded; a wait that expires sets ABCS_DEV_TIMEOUT
// and an abort flag that ends every role, and the CTA frees its tensor
// memory before it leaves.
// ---------------------------------------------------------------------------
constexpr int T5_TW = 128, T5_IW = T5_TW + 2;
constexpr int T5_EPI_WARPS = 8, T5_THREADS = 32 * (2 + T5_EPI_WARPS);
// shared layout of a tile height TH: NBUF input tiles, the weights, misc
template <int TH>
struct T5Tile {
    static constexpr int IH = TH + 2;
    static constexpr uint32_t PLANE = IH * T5_IW * 16;     // bytes of one 8-channel plane of a tile
    static constexpr uint32_t TILE = 4 * PLANE;            // 4 planes x IH rows x 130 pixels
    static constexpr int NBUF = TH == 4 ? 3 : 2;
    static constexpr uint32_t WOFF = NBUF * TILE;          // weights after the tiles
    static constexpr uint32_t MISC = WOFF + 9 * kC * kC * 2;   // mbarriers, tensor-memory address, abort flag
    static constexpr size_t SMEM = MISC + 128;
    static_assert(PLANE % 16 == 0 && TILE % 128 == 0, "bulk-copy destinations stay 16-byte aligned");
    static_assert(SMEM <= 232448 && NBUF <= 3 && 2 * TH * 32 <= 512, "tcgen05 conv shared / tensor memory layout");
};
// mbarriers in the misc area: full[3], empty[3], acc_full[2], acc_empty[2]
constexpr uint32_t T5_FULL = 0, T5_EMPTY = 24, T5_AFULL = 48, T5_AEMPTY = 64, T5_SLOT = 80, T5_ABORT = 84;

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t t5_idesc(uint32_t n) { return umma_idesc_f16(n, true); }

ABCS_D void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// NC = 32: a 32 -> 32 layer (bias, ReLU, BF16 chunk-planar out).  NC = 16: the last
// layer; B columns 0 and 1 hold the BF16 hi and lo parts of its FP32
// weights (the rest zero) and the epilogue writes mode 0: r - 255 (c0 + c1
// + b), mode 1: c0 + c1 + b, in FP32.
template <int NC, int TH>
__global__ void __launch_bounds__(T5_THREADS, 1) conv32_tc5_kernel(const __nv_bfloat16* __restrict__ in,
                                                                   int n, int H, int W,
                                                                   const __nv_bfloat16* __restrict__ wts,
                                                                   const float* __restrict__ bias,
                                                                   __nv_bfloat16* __restrict__ out,
                                                                   const float* __restrict__ r_in, int mode,
                                                                   float* __restrict__ fout,
                                                                   uint32_t* status) {
    // weights: per dx, per 16-byte K chunk, rows n = dy NC + co (the three dy taps side by side in N)
    using L = T5Tile<TH>;
    constexpr uint32_t WCHUNK = 3 * NC * 16, WDX = 4 * WCHUNK, TMEM_COLS = 2 * TH * NC;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t sb = smem_u32(smem), mb = sb + L::MISC;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::MISC + T5_SLOT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::MISC + T5_ABORT);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int tx = (W + T5_TW - 1) / T5_TW, ty = (H + TH - 1) / TH, per_img = tx * ty;
    const int ntiles = per_img * n;
    const int G = gridDim.x;
    if ((int)blockIdx.x >= ntiles) return;
    const int my_n = (ntiles - (int)blockIdx.x + G - 1) / G;
    auto origin = [&](int j, int& k, int& y0, int& x0) {
        const int tile = (int)blockIdx.x + j * G;
        k = tile / per_img;
        const int rem = tile - k * per_img, by = rem / tx;
        y0 = by * TH;
        x0 = (rem - by * tx) * T5_TW;
    };

    // the layer's weights (tap, 16-byte chunk c = ci 8c .. 8c+7, row co), barriers, tensor memory
    for (int i = t; i < 9 * NC * 4; i += T5_THREADS) {
        const int tap = i / (NC * 4), co = (i >> 2) % NC, c = i & 3, dy = tap / 3, dx = tap % 3;
        cp_async16_zfill(smem + L::WOFF + dx * WDX + c * WCHUNK + (dy * NC + co) * 16,
                         wts + (tap * NC + co) * kC + c * 8, true);
    }
    cp_async_commit();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (t == 0) {
        for (int b = 0; b < L::NBUF; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb + T5_FULL + 8 * b) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb + T5_EMPTY + 8 * b) : "memory");
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb + T5_AFULL + 8 * a) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb + T5_AEMPTY + 8 * a),
                         "r"(T5_EPI_WARPS)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort_flag = 0;
    }
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    const uint32_t tmem = *tmem_slot;
    griddep_wait();

    if (warp == 0) {
        // ---- producer: run q = lane + 32 u (plane q / IH, input row q % IH) of
        // a tile is one bulk copy of its in-image pixels (a contiguous run of
        // the chunk-planar activations); pixels outside the image are zeroed here
        constexpr int RUNS = 4 * L::IH, NP = (RUNS + 31) / 32;
        for (int j = 0; j < my_n; ++j) {
            const int b = j % L::NBUF;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(mb + T5_EMPTY + 8 * b, ((j / L::NBUF) & 1) ^ 1, abort_flag, status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            int k, y0, x0;
            origin(j, k, y0, x0);
            const int xa = x0 - 1 > 0 ? x0 - 1 : 0, xb = x0 + T5_TW + 1 < W ? x0 + T5_TW + 1 : W;
            uint32_t nb[NP], total = 0;
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                const int q = lane + 32 * u, c = q / L::IH, i = q - c * L::IH, y = y0 - 1 + i;
                const bool mine = q < RUNS;
                const bool row_in = mine && y >= 0 && y < H && xb > xa;
                nb[u] = row_in ? (uint32_t)(xb - xa) * 16u : 0u;
                total += nb[u];
                if (mine) {
                    const uint32_t seg = sb + b * L::TILE + c * L::PLANE + i * T5_IW * 16;
                    const int za = row_in ? xa - (x0 - 1) : T5_IW, zb = row_in ? xb - (x0 - 1) : T5_IW;
                    for (int p = 0; p < za; ++p)      // left halo (and whole rows outside the image)
                        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(seg + 16 * p), "r"(0) : "memory");
                    for (int p = zb; p < T5_IW; ++p)  // right halo
                        asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(seg + 16 * p), "r"(0) : "memory");
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            const uint32_t full = mb + T5_FULL + 8 * b;
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(full), "r"(total)
                             : "memory");
            __syncwarp();
#pragma unroll
            for (int u = 0; u < NP; ++u) {
                if (nb[u]) {
                    const int q = lane + 32 * u, c = q / L::IH, i = q - c * L::IH, y = y0 - 1 + i;
                    const uint32_t seg = sb + b * L::TILE + c * L::PLANE + i * T5_IW * 16;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                            seg + (uint32_t)(xa - (x0 - 1)) * 16u),
                        "l"(in + act_off(k, y, xa, 8 * c, H, W)), "r"(nb[u]), "r"(full)
                        : "memory");
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            const uint64_t bdesc0 = umma_desc(sb + L::WOFF, WCHUNK, 128);
            for (int j = 0; j < my_n; ++j) {
                const int b = j % L::NBUF, a = j & 1;
                if (!mbar_wait(mb + T5_FULL + 8 * b, (j / L::NBUF) & 1, abort_flag, status)) break;
                if (!mbar_wait(mb + T5_AEMPTY + 8 * a, ((j >> 1) & 1) ^ 1, abort_flag, status)) break;
                tc5_fence_after();
                const uint64_t adesc0 = umma_desc(sb + b * L::TILE, L::PLANE, 128);
                // output row r accumulates at column (T - 1 - r) NC, so input row i
                // feeds rows i - dy_lo .. i - dy_hi through one MMA whose N
                // covers the dy taps side by side; row r starts fresh at i = r
                const uint32_t d0 = tmem + (uint32_t)(a * (TH * NC));
#pragma unroll
                for (int i = 0; i < L::IH; ++i) {
                    const int dy_lo = i - (TH - 1) > 0 ? i - (TH - 1) : 0, dy_hi = i < 2 ? i : 2;
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint64_t ad = adesc0 + (uint64_t)(((i * T5_IW + dx) * 16 + 2 * h * L::PLANE) >> 4);
                            const uint32_t bb = dx * WDX + 2 * h * WCHUNK;
                            if (dx == 0 && h == 0 && dy_lo == 0) {
                                umma_bf16(d0 + (TH - 1 - i) * NC, ad, bdesc0 + (bb >> 4), t5_idesc(NC), 0);
                                if (dy_hi >= 1)
                                    umma_bf16(d0 + (TH - i) * NC, ad, bdesc0 + ((bb + NC * 16) >> 4),
                                              t5_idesc(dy_hi * NC), 1);
                            } else {
                                umma_bf16(d0 + (TH - 1 - i + dy_lo) * NC, ad,
                                          bdesc0 + ((bb + dy_lo * NC * 16) >> 4),
                                          t5_idesc((dy_hi - dy_lo + 1) * NC), 1);
                            }
                        }
                    }
                }
                umma_commit(mb + T5_EMPTY + 8 * b);        // the input buffer is free once these complete
                umma_commit(mb + T5_AFULL + 8 * a);        // the accumulators are ready
            }
        }
    } else {
        // ---- epilogue
        const int e = warp - 2, lg = warp & 3, r0 = e >> 2;
        float bz[NC == 32 ? 32 : 1];
#pragma unroll
        for (int c = 0; c < (NC == 32 ? 32 : 1); ++c) bz[c] = __ldg(bias + c);
        for (int j = 0; j < my_n; ++j) {
            const int a = j & 1;
            if (!mbar_wait(mb + T5_AFULL + 8 * a, (j >> 1) & 1, abort_flag, status)) break;
            tc5_fence_after();
            int k, y0, x0;
            origin(j, k, y0, x0);
            const int x = x0 + 32 * lg + lane;
#pragma unroll
            for (int r = r0; r < TH; r += 2) {
                const uint32_t ta = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(a * (TH * NC) + (TH - 1 - r) * NC);
                const int y = y0 + r;
                if constexpr (NC == 32) {
                    uint32_t v[32];
                    tmem_ld32(ta, v);
                    if (x < W && y < H) {
                        uint32_t o[16];
#pragma unroll
                        for (int c = 0; c < 16; ++c)
                            o[c] = pack_bf16_relu(__uint_as_float(v[2 * c]) + bz[2 * c],
                                                  __uint_as_float(v[2 * c + 1]) + bz[2 * c + 1]);
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            *reinterpret_cast<uint4*>(out + act_off(k, y, x, 8 * c, H, W)) =
                                make_uint4(o[4 * c], o[4 * c + 1], o[4 * c + 2], o[4 * c + 3]);
                    }
                } else {
                    uint32_t v0, v1;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n"
                                 : "=r"(v0), "=r"(v1)
                                 : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (x < W && y < H) {
                        const float a_ = __uint_as_float(v0) + __uint_as_float(v1) + bz[0];
                        const int64_t o = ((int64_t)k * H + y) * W + x;
                        fout[o] = mode == 0 ? __ldg(r_in + o) - 255.f * a_ : a_;
                    }
                }
            }
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mb + T5_AEMPTY + 8 * a) : "memory");
        }
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

template <int NC, int TH>
static cudaError_t tc5_launch(const __nv_bfloat16* in, int n, int H, int W, const __nv_bfloat16* wts,
                              const float* bias, __nv_bfloat16* out, const float* r_in, int mode, float* fout,
                              uint32_t* status, cudaStream_t s) {
    using L = T5Tile<TH>;
    cudaError_t e =
        cudaFuncSetAttribute((conv32_tc5_kernel<NC, TH>), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    int dev, sms;
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) return e;
    const int64_t tiles = (int64_t)((W + T5_TW - 1) / T5_TW) * ((H + TH - 1) / TH) * n;
    const int grid = (int)(tiles < sms ? tiles : sms);
    return launch_pdl((conv32_tc5_kernel<NC, TH>), dim3(grid), dim3(T5_THREADS), L::SMEM, s, in, n, H, W, wts, bias,
                      out, r_in, mode, fout, status);
}

static cudaError_t conv32_tc5_launch(const __nv_bfloat16* in, int n, int H, int W, const __nv_bfloat16* wts,
                                     const float* bias, __nv_bfloat16* out, uint32_t* status, cudaStream_t s) {
    return tc5_launch<32, 4>(in, n, H, W, wts, bias, out, nullptr, 0, nullptr, status, s);
}

template <int EPI>
static cudaError_t conv32_launch(const __nv_bfloat16* in, int n, int H, int W, const __nv_bfloat16* wts,
                                 const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(conv32_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kConvSmem);
    int dev, sms, per_sm;
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv32_kernel<EPI>, 256, kConvSmem);
    if (e) return e;
    const int64_t tiles = (int64_t)((W + TW - 1) / TW) * ((H + TH - 1) / TH) * n;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(tiles < cap ? tiles : cap);
    return launch_pdl(conv32_kernel<EPI>, dim3(grid), dim3(256), kConvSmem, s, in, n, H, W, wts, bias, mask, out);
}

static cudaError_t conv32(int epi, const __nv_bfloat16* in, int n, int H, int W, const __nv_bfloat16* wts,
                          const float* bias, const __nv_bfloat16* mask, __nv_bfloat16* out, cudaStream_t s) {
    return epi == 0 ? conv32_launch<0>(in, n, H, W, wts, bias, mask, out, s)
                    : conv32_launch<1>(in, n, H, W, wts, bias, mask, out, s);
}

// Forward through layers 0..6 into act[0..6] (each n*H*W*32 bf16), then the
// last layer into out (mode 0: denoised image, mode 1: network output n).
cudaError_t cnn_forward(const void* packed, const float* r, const float* sigma, const float* dens, const float* tau,
                        float tau0, int n, int H, int W, void* act_buf, int keep_all, int mode, float* out,
                        uint32_t* status, cudaStream_t s) {
    const CnnPacked* P = static_cast<const CnnPacked*>(packed);
    const int64_t plane = (int64_t)n * H * W * kC;
    __nv_bfloat16* act = static_cast<__nv_bfloat16*>(act_buf);
    auto A = [&](int l) { return act + (keep_all ? l : (l & 1)) * plane; };
    int dev, sms, per_sm;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cnn_first_tc_kernel, 256, 0);
    if (e) return e;
    const int64_t tiles = (int64_t)((W + TW - 1) / TW) * ((H + TH - 1) / TH) * n;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    e = launch_pdl(cnn_first_tc_kernel, dim3((unsigned)(tiles < cap ? tiles : cap)), dim3(256), 0, s, r, sigma,
                   dens, tau, tau0, n, H, W, P, A(0));
    for (int l = 1; l <= kMid && !e; ++l)
        e = conv32_tc5_launch(A(l - 1), n, H, W, &P->wc[l - 1][0][0][0], &P->bm[l - 1][0], A(l), status, s);
    if (e) return e;
    return tc5_launch<16, 8>(A(kMid), n, H, W, &P->w7t[0][0][0], &P->b7, nullptr, r, mode, out, status, s);
}

// Loss and gradients (FP32, parameter layout) of a batch of n crops.
// Workspace: act (7 planes), gbuf (2 planes), gn (n*H*W floats), parts.
cudaError_t cnn_grad(const void* packed, const float* r, const float* clean, const float* sigma, const float* dens,
                     const float* tau, int n, int H, int W, void* ws, float* grad, float* loss, uint32_t* status,
                     cudaStream_t s) {
    const CnnPacked* P = static_cast<const CnnPacked*>(packed);
    const int64_t px = (int64_t)n * H * W, plane = px * kC;
    char* w = static_cast<char*>(ws);
    __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(w);
    __nv_bfloat16* gb = act + 7 * plane;                         // 2 gradient planes
    float* nout = reinterpret_cast<float*>(gb + 2 * plane);
    float* gn = nout + px;
    const int nparts = 304;
    float* part = gn + px;                                       // nparts * (kWm + kBm)
    double* lpart = reinterpret_cast<double*>(part + (size_t)nparts * (kWm + kBm));
    cudaError_t e = cnn_forward(packed, r, sigma, dens, tau, 0.f, n, H, W, act, 1, 1, nout, status, s);
    if (e) return e;
    cnn_loss_kernel<<<256, 256, 0, s>>>(nout, r, clean, px, gn, lpart);
    reduce_loss_kernel<<<1, 32, 0, s>>>(lpart, 256, loss);
    dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH, n);
    const int tiles = grid.x * grid.y * n;
    const int np = tiles < nparts ? tiles : nparts;
    // last layer
    const size_t smem_l = (size_t)IH * IW * 33 * 4;
    if ((e = cudaFuncSetAttribute(wgrad_last_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l))) return e;
    wgrad_last_kernel<<<np, 256, smem_l, s>>>(act + kMid * plane, gn, n, H, W, part);
    reduce_parts_kernel<<<(kW7 + kB7 + 255) / 256, 256, 0, s>>>(part, np, kW7 + kB7, grad + param_off_w(7));
    cnn_last_bwd_kernel<<<grid, 256, 0, s>>>(gn, act + kMid * plane, H, W, P, gb);
    // mid layers, l = 6 .. 1: g_l (pre-activation grad) in gb[cur]
    const size_t smem_w = (size_t)(IH * IW + TH * TW) * 33 * 4;
    if ((e = cudaFuncSetAttribute(wgrad32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w))) return e;
    int cur = 0;
    for (int l = kMid; l >= 1; --l) {
        __nv_bfloat16* g = gb + cur * plane;
        wgrad32_kernel<<<np, 256, smem_w, s>>>(act + (l - 1) * plane, g, n, H, W, part);
        reduce_parts_kernel<<<(kWm + kBm + 255) / 256, 256, 0, s>>>(part, np, kWm + kBm, grad + param_off_w(l));
        // input gradient, masked by the ReLU of layer l-1's output
        e = conv32(1, g, n, H, W, &P->wd[l - 1][0][0][0], nullptr, act + (l - 1) * plane, gb + (1 - cur) * plane, s);
        if (e) return e;
        cur = 1 - cur;
    }
    wgrad_first_kernel<<<np, 256, 0, s>>>(r, sigma, dens, tau, 0.f, gb + cur * plane, n, H, W, part);
    reduce_parts_kernel<<<(kW0 + kB0 + 255) / 256, 256, 0, s>>>(part, np, kW0 + kB0, grad);
    return cudaGetLastError();
}

size_t cnn_grad_ws_bytes(int n, int H, int W) {
    const int64_t px = (int64_t)n * H * W, plane = px * kC;
    return (size_t)(9 * plane) * 2 + (size_t)(2 * px) * 4 + (size_t)304 * (kWm + kBm) * 4 + 256 * 8 + 1024;
}

cudaError_t cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(params, grad, m, v, kParams, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace abcs
