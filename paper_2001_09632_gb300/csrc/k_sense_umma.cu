// Sensing on the 5th-generation tensor cores (B = 16): the measurements of
// a tile of 32 blocks as ONE GEMM against the zigzag-ordered DCT basis.
//
// With phi_k the basis image of zigzag rank k (phi_k[16 r + c] =
// D[u_k][r] D[v_k][c], Eq. 1 and the zigzag order of Sec. IV), block b's
// rank-k measurement (a row of Eq. 26's A applied to the block) is
//   y_b[k] = sum_p phi_k[p] x_b[p].
// For a tile of NT = 64 blocks and the ranks of one half h (k = 128 h + m):
//   Y_h[m][n] = sum_p 16 phi_{128 h + m}[p] x_n[p] / 16
//   (M = 128 ranks, N = 64 blocks, K = 256 pixels)
// The pixels (uint8) are exact in FP16 and BF16, so only the constant
// operand is split: 16 phi = hi + lo (hi + lo = 16 phi to about 22 bits in
// FP16x2 / 16 bits in BF16x2, one BF16 word for plain BF16), and each half
// costs two K = 256 products (hi and lo) accumulated in FP32 in tensor
// memory.  The factor 16 keeps the FP16 low words out of the subnormal
// range; it is divided out exactly in the epilogue.
//
// Tensor memory (512 columns of 32 bits, 128 lanes):
//   [0, 128)    A of half 0, hi words (lane m = rank m, column c = pixels 2c, 2c + 1)
//   [128, 256)  A of half 0, lo words
//   [256, 384)  accumulator of MMA issuer 0: half 0 (64 blocks), then half 1
//   [384, 512)  accumulator of MMA issuer 1
// Half 1's A (ranks 128 .. 255, hi and lo) is a shared-memory operand.
// Half 1 is computed only for tiles whose largest count exceeds 128 (a
// third of the tiles at subrate 0.3).
//
// A single thread issues one tcgen05.mma about every 50 cycles whatever N
// is, while an M = 128, N = 64, K = 16 product takes the tensor pipe 32
// cycles, so two issuing warps take alternate tiles (each with its own B
// stage and accumulator) and keep the pipe busy.
//
// Roles (19 warps, one CTA per SM, tiles c, c + G, c + 2G, ...):
//   warps 0, 1  MMA issuers (lane 0); warp 0 also allocates tensor memory
//               and loads the operand table (bulk copies)
//   warp 2      metadata, up to four tiles ahead: counts, global offsets
//               (image-local offset + image base) and largest count
//   warps 3-10  converters: 16-byte global loads of pixel rows one tile
//               ahead (a warp reads 512 contiguous bytes of a row), FP16 /
//               BF16 pairs into the tile's K-major B stage (conflict free)
//   warps 11-18 epilogue: warp w reads lanes 32 (w % 4) .. (32 ranks) of
//               32 of the tile's columns (blocks) and stores rank k of block
//               n to y[offset_n + k] when k < m_n (a warp store covers 32
//               consecutive coefficients of one block), predicated, without
//               branches; it also writes the global offsets
// The pixel loads and the half-0 products of the first tiles need no
// allocation result, so they run while the pilot kernel finishes (PDL).
// Every wait is bounded: on expiry ABCS_DEV_TIMEOUT is set and an abort flag
// ends every role; MMAs in flight are drained before the CTA frees its
// tensor memory.
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "abcs_common.cuh"
#include "umma.cuh"

namespace abcs {
ABCS_TU_TABLES(su)
}  // namespace abcs

namespace abcs {

namespace {

constexpr int kSP16 = ABCS_TC_FP16X2, kSPB16 = ABCS_TC_BF16X2, kSPB1 = ABCS_TC_BF16;

template <int P>
__host__ __device__ constexpr int su_pidx() { return P == kSP16 ? 0 : (P == kSPB16 ? 1 : 2); }

template <int P>
ABCS_D uint32_t su_pk(float a, float b) {     // a -> low half, b -> high half
    if constexpr (P == kSP16) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

template <int P>
ABCS_D void su_unpk(uint32_t v, float& a, float& b) {
    if constexpr (P == kSP16) {
        const __half2 h = *reinterpret_cast<const __half2*>(&v);
        a = __low2float(h);
        b = __high2float(h);
    } else {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&v);
        a = __low2float(h);
        b = __high2float(h);
    }
}

// (a, b) in FP64 -> hi pair and lo (residual) pair
template <int P>
ABCS_D void su_split(double a, double b, uint32_t& hi, uint32_t& lo) {
    hi = su_pk<P>((float)a, (float)b);
    float ha, hb;
    su_unpk<P>(hi, ha, hb);
    lo = su_pk<P>((float)(a - ha), (float)(b - hb));
}

constexpr int NT = 64;                 // blocks per tile (the MMA's N)
constexpr int SU_I = 4;                // metadata slots
constexpr float SU_SCALE = 16.f;
constexpr uint32_t SU_PART = 65536;    // bytes of one operand-table part
constexpr uint32_t SU_STAGE = NT * 512;   // 32 K chunks of NT rows x 16 bytes
constexpr int SU_CONV = 8;             // converter warps
constexpr int SU_EPI = 8;              // epilogue warps (two per tensor-memory lane quarter)
// warp roles
constexpr int W_MMA0 = 0, W_MMA1 = 1, W_META = 2, W_CONV = 3, W_EPI = W_CONV + SU_CONV;
constexpr int SU_THREADS = 32 * (W_EPI + SU_EPI);

struct SuInfo {
    uint32_t pk[NT];   // per block: offset relative to base (low 16 bits) | count << 16
    int64_t base;      // global offset of the tile's first block
    int kmax;          // largest count of the tile
    int pad;
};
static_assert(sizeof(SuInfo) % 16 == 0, "metadata slots stay 16-byte aligned");

constexpr uint32_t SU_OFF_A1HI = 0;                               // also staging of the table parts
constexpr uint32_t SU_OFF_A1LO = SU_PART;
constexpr int SU_S = 3;                // B stages (tile j uses stage j % 3)
constexpr uint32_t SU_OFF_B = 2 * SU_PART;
constexpr uint32_t SU_OFF_INFO = SU_OFF_B + SU_S * SU_STAGE;
constexpr uint32_t SU_OFF_BAR = SU_OFF_INFO + SU_I * sizeof(SuInfo);
// mbarriers
constexpr uint32_t SU_BF = 0, SU_BE = 24, SU_ACCF = 48, SU_ACCE = 64, SU_INF = 80, SU_INE = SU_INF + 8 * SU_I,
                   SU_TABF = SU_INE + 8 * SU_I, SU_TABE = SU_TABF + 8, SU_TABR = SU_TABE + 8, SU_DRAIN = SU_TABR + 8,
                   SU_NBAR = SU_DRAIN + 16;
constexpr uint32_t SU_OFF_MISC = SU_OFF_BAR + SU_NBAR;            // tensor-memory address, abort flag
constexpr size_t SU_SMEM = SU_OFF_MISC + 16;
static_assert(SU_OFF_B % 1024 == 0 && SU_OFF_INFO % 16 == 0 && SU_OFF_BAR % 8 == 0, "shared layout");
static_assert(SU_SMEM <= 232448, "shared memory of the tensor-memory sensing kernel");

// Operand table per precision, four 64 KB parts of 16 phi (rows = ranks of
// a half, K = pixels):
//   parts 0, 1: tensor-memory words of half 0, hi and lo:
//               word [c][m] = (A[m][2c], A[m][2c + 1])
//   parts 2, 3: half 1 hi and lo as their shared-memory K-major images:
//               byte 2048 kc + 16 m + 2 e = A[m][8 kc + e]
__device__ __align__(16) uint32_t g_sphi[3][4][SU_PART / 4];

template <int P>
ABCS_D void sphi_setup_p(int half, int m, int c) {
    const int z = zz_pos<16>(128 * half + m);
    const int u = z >> 4, v = z & 15;
    double a[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int p = 2 * c + e, r = p >> 4, col = p & 15;
        a[e] = (double)SU_SCALE * Dd<16>(u, r) * Dd<16>(v, col);
    }
    uint32_t hi, lo;
    su_split<P>(a[0], a[1], hi, lo);
    uint32_t(*t)[SU_PART / 4] = g_sphi[su_pidx<P>()];
    if (half == 0) {
        t[0][c * 128 + m] = hi;
        t[1][c * 128 + m] = lo;
    } else {
        // pixels 2c, 2c + 1: chunk kc = 2c / 8, word (2c % 8) / 2 of row m
        t[2][(c >> 2) * 512 + m * 4 + (c & 3)] = hi;
        t[3][(c >> 2) * 512 + m * 4 + (c & 3)] = lo;
    }
}

__global__ void sphi_setup_kernel() {     // grid (128 columns, 2 halves), block 128 (ranks)
    const int c = blockIdx.x, half = blockIdx.y, m = threadIdx.x;
    sphi_setup_p<kSP16>(half, m, c);
    sphi_setup_p<kSPB16>(half, m, c);
    sphi_setup_p<kSPB1>(half, m, c);
}

// D (tensor memory) (+)= A (tensor memory) * B (shared-memory descriptor);
// the accumulate flag is a compile-time constant
template <int ACC>
ABCS_D void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "n"(ACC));
}

// D (tensor memory) (+)= A (shared-memory descriptor) * B (shared-memory descriptor)
template <int ACC>
ABCS_D void mma_sa(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "n"(ACC));
}

// y[i] = v when pred, as one predicated store (no branch around it)
ABCS_D void st_pred(float* p, float v, bool pred) {
    asm volatile("{\n.reg .pred q;\nsetp.ne.b32 q, %2, 0;\n@q st.global.f32 [%0], %1;\n}\n" ::"l"(p), "f"(v),
                 "r"((int)pred));
}

// two pixels (bytes 2 sel, 2 sel + 1 of w) as an operand pair; exact
template <int P>
ABCS_D uint32_t su_px2(uint32_t w, int sel) {
    if constexpr (P == kSP16) {
        // 0x64XX as FP16 is 1024 + XX exactly; subtract 1024
        const uint32_t v = __byte_perm(w, 0x64646464u, sel ? 0x4342 : 0x4140);
        const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&v),
                                  __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        return su_pk<P>((float)((w >> (16 * sel)) & 0xFF), (float)((w >> (16 * sel + 8)) & 0xFF));
    }
}

// block b of the batch (b < 2^31) -> image k, block row bi, block column bj
ABCS_D void su_coords(const ImgGeom& g, int64_t b, int& k, int& bi, int& bj) {
    const int bb = (int)b, nB = (int)g.n_blocks;
    k = bb / nB;
    const int i = bb - k * nB;
    bi = i / g.nbw;
    bj = i - bi * g.nbw;
}

template <int P>
__global__ void __launch_bounds__(SU_THREADS, 1) sense_umma_kernel(SenseArgs a, int64_t ntot) {
    extern __shared__ __align__(1024) unsigned char su_smem[];
    unsigned char* smem = su_smem;
    constexpr bool kSplit = P != kSPB1;
    constexpr uint32_t IDESC = umma_idesc_f16(NT, P != kSP16);
    const uint32_t sb = smem_u32(smem), bar = sb + SU_OFF_BAR;
    SuInfo* info = reinterpret_cast<SuInfo*>(smem + SU_OFF_INFO);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + SU_OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + SU_OFF_MISC + 4);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int G = gridDim.x;
    const int64_t T = (ntot + NT - 1) / NT;
    const int my_n = blockIdx.x < T ? (int)((T - blockIdx.x + G - 1) / G) : 0;
    const ImgGeom& g = a.g;
    auto tile_b0 = [&](int j) { return ((int64_t)blockIdx.x + (int64_t)j * G) * NT; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (t == 32) {
        for (int i = 0; i < SU_S; ++i) {
            mbar_init(bar + SU_BF + 8 * i, SU_CONV);
            mbar_init(bar + SU_BE + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar + SU_ACCF + 8 * i, 1);
            mbar_init(bar + SU_ACCE + 8 * i, SU_EPI);
            mbar_init(bar + SU_DRAIN + 8 * i, 1);
        }
        for (int i = 0; i < SU_I; ++i) {
            mbar_init(bar + SU_INF + 8 * i, 1);
            mbar_init(bar + SU_INE + 8 * i, SU_EPI);
        }
        mbar_init(bar + SU_TABF, 1);
        mbar_init(bar + SU_TABE, SU_EPI);
        mbar_init(bar + SU_TABR, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort_flag = 0;
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == W_MMA0 || warp == W_MMA1) {
        // ---- operand table (issuer 0), then the MMA issuers: issuer i takes
        // the tiles j = i mod 2 with B stage i and accumulator i
        const int me = warp - W_MMA0;
        if (lane == 0) {
            bool alive = true;
            if (me == 0) {
                const uint32_t* tab = &g_sphi[su_pidx<P>()][0][0];
                // half 0 (parts 0, 1) staged in the half-1 regions and copied
                // into tensor memory by the epilogue warps; then half 1
                // (parts 2, 3) lands in its regions
                const uint32_t n0 = kSplit ? 2 * SU_PART : SU_PART;
                mbar_arrive_tx(bar + SU_TABF, n0);
                bulk_g2s(sb + SU_OFF_A1HI, tab, SU_PART, bar + SU_TABF);
                if (kSplit) bulk_g2s(sb + SU_OFF_A1LO, tab + SU_PART / 4, SU_PART, bar + SU_TABF);
                alive = mbar_wait(bar + SU_TABF, 0, abort_flag, a.status) &&
                        mbar_wait(bar + SU_TABE, 0, abort_flag, a.status);
                if (alive) {
                    mbar_arrive_tx(bar + SU_TABF, n0);
                    bulk_g2s(sb + SU_OFF_A1HI, tab + 2 * (SU_PART / 4), SU_PART, bar + SU_TABF);
                    if (kSplit) bulk_g2s(sb + SU_OFF_A1LO, tab + 3 * (SU_PART / 4), SU_PART, bar + SU_TABF);
                    alive = mbar_wait(bar + SU_TABF, 1, abort_flag, a.status);
                }
                if (alive) mbar_arrive(bar + SU_TABR);
            }
            // both issuers: half 0 in tensor memory (the epilogue's copies) and
            // half 1 in shared memory are ready
            if (alive && !mbar_wait(bar + SU_TABE, 0, abort_flag, a.status)) alive = false;
            if (alive && !mbar_wait(bar + SU_TABR, 0, abort_flag, a.status)) alive = false;
            tc5_fence_after();
            const uint32_t d0 = tmem + 256 + 128 * me, d1 = d0 + 64;
            const uint64_t ah0 = umma_desc(sb + SU_OFF_A1HI, 2048, 128), al0 = umma_desc(sb + SU_OFF_A1LO, 2048, 128);
            for (int j = me, u = 0; j < my_n && alive; j += 2, ++u) {
                const int is = j % SU_I, st = j % SU_S;
                const uint64_t bd0 = umma_desc(sb + SU_OFF_B + st * SU_STAGE, NT * 16, 128);
                if (!mbar_wait(bar + SU_ACCE + 8 * me, (u & 1) ^ 1, abort_flag, a.status)) break;
                if (!mbar_wait(bar + SU_BF + 8 * st, (j / SU_S) & 1, abort_flag, a.status)) break;
                tc5_fence_after();
                // K step ks: pixel row ks = B chunks 2 ks, 2 ks + 1 (ks * 2 * NT * 16 bytes,
                // i.e. ks * 2 * NT in the descriptor's 16-byte address units)
                mma_ta<0>(d0, tmem, bd0, IDESC);
                if constexpr (kSplit) mma_ta<1>(d0, tmem + 128, bd0, IDESC);
#pragma unroll
                for (int ks = 1; ks < 16; ++ks) {
                    const uint64_t bd = bd0 + (uint64_t)(ks * 2 * NT);
                    mma_ta<1>(d0, tmem + 8 * ks, bd, IDESC);
                    if constexpr (kSplit) mma_ta<1>(d0, tmem + 128 + 8 * ks, bd, IDESC);
                }
                // half 1 only where some block of the tile needs ranks >= 128
                if (!mbar_wait(bar + SU_INF + 8 * is, (j / SU_I) & 1, abort_flag, a.status)) break;
                if (info[is].kmax > 128) {
                    mma_sa<0>(d1, ah0, bd0, IDESC);
                    if constexpr (kSplit) mma_sa<1>(d1, al0, bd0, IDESC);
#pragma unroll
                    for (int ks = 1; ks < 16; ++ks) {
                        const uint64_t bd = bd0 + (uint64_t)(ks * 2 * NT);
                        mma_sa<1>(d1, ah0 + (uint64_t)(ks * 256), bd, IDESC);
                        if constexpr (kSplit) mma_sa<1>(d1, al0 + (uint64_t)(ks * 256), bd, IDESC);
                    }
                }
                umma_commit(bar + SU_BE + 8 * st);        // the stage is free once these complete
                umma_commit(bar + SU_ACCF + 8 * me);      // the tile's accumulator is ready
            }
            umma_commit(bar + SU_DRAIN + 8 * me);
            mbar_drain(bar + SU_DRAIN + 8 * me, 0, a.status);
        }
        __syncwarp();
    } else if (warp == W_META) {
        // ---- metadata, up to SU_I tiles ahead of the epilogue: lane = blocks
        // lane, lane + 32.  Global offset = image-local offset + the image's
        // base, derived from the per-image totals: a running base of the
        // tile's first image (the gap to the next tile summed by the warp)
        // plus a 64-wide prefix of the totals of the tile's images.
        griddep_wait();
        int kc = 0;
        int64_t basec = 0;
        for (int j = 0; j < my_n; ++j) {
            const int is = j % SU_I;
            if (j >= SU_I) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(bar + SU_INE + 8 * is, ((j / SU_I) & 1) ^ 1, abort_flag, a.status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            }
            const int64_t b0 = tile_b0(j);
            const int n = (int)(ntot - b0 < NT ? ntot - b0 : NT);
            const int kseg = (int)(b0 / g.n_blocks);
            {
                int64_t v = 0;
                for (int k = kc + lane; k < kseg; k += 32) v += __ldg(a.img_total + k);
                basec += warp_sum(v);
                kc = kseg;
            }
            const int64_t ta = kseg + lane < g.n_img ? __ldg(a.img_total + kseg + lane) : 0;
            const int64_t tb = kseg + 32 + lane < g.n_img ? __ldg(a.img_total + kseg + 32 + lane) : 0;
            int64_t ia = ta, ib = tb;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
                if (lane >= o) {
                    ia += ua;
                    ib += ub;
                }
            }
            ib += __shfl_sync(0xffffffffu, ia, 31);
            const int64_t ea = ia - ta, eb = ib - tb;     // bases of images kseg + lane, kseg + 32 + lane (minus basec)
            int m[2];
            int64_t off[2];
            bool bad = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                m[h] = 0;
                off[h] = 0;
                int d = 0;
                if (i < n) {
                    int k, bi, bj;
                    su_coords(g, b0 + i, k, bi, bj);
                    d = k - kseg;                      // 0 .. 63
                    m[h] = __ldg(a.counts + b0 + i);
                    off[h] = __ldg(a.offsets + b0 + i);
                }
                const int64_t xa = __shfl_sync(0xffffffffu, ea, d & 31), xb = __shfl_sync(0xffffffffu, eb, d & 31);
                if (i < n) off[h] += basec + (d < 32 ? xa : xb);
            }
            const int64_t base = __shfl_sync(0xffffffffu, off[0], 0);
            SuInfo& I = info[is];
            int km = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = lane + 32 * h;
                int64_t rel = off[h] - base;
                if (i < n && (m[h] < 0 || m[h] > 256 || rel < 0 || rel + m[h] > NT * 256)) {
                    bad = true;
                    m[h] = 0;
                    rel = 0;
                }
                if (i >= n) {
                    m[h] = 0;
                    rel = 0;
                }
                I.pk[i] = (uint32_t)rel | ((uint32_t)m[h] << 16);
                km = max(km, m[h]);
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(a.status, ABCS_DEV_BADCOUNT);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
            if (lane == 0) {
                I.base = base;
                I.kmax = km;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_INF + 8 * is);
        }
    } else if (warp < W_EPI) {
        // ---- converters: warp c takes blocks lane + 32 (c & 1) of the tile
        // and pixel rows (c >> 1) + 4 i; global 16-byte loads one tile ahead,
        // FP16 / BF16 pairs into the K-major B stage of the tile's issuer
        const int c = warp - W_CONV, nb = lane + 32 * (c & 1), r0 = c >> 1;
        uint4 cur[4], nxt[4];
        auto load = [&](int j, uint4 (&v)[4]) {
            const int64_t b0 = tile_b0(j);
            if (b0 + nb < ntot) {
                int k, bi, bj;
                su_coords(g, b0 + nb, k, bi, bj);
                const uint8_t* src = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * 16 + r0) * g.pitch + bj * 16;
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = __ldg(reinterpret_cast<const uint4*>(src + (int64_t)(4 * i) * g.pitch));
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] = make_uint4(0, 0, 0, 0);
            }
        };
        if (my_n > 0) load(0, cur);
        for (int j = 0; j < my_n; ++j) {
            if (j + 1 < my_n) load(j + 1, nxt);
            const int st = j % SU_S;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar + SU_BE + 8 * st, ((j / SU_S) & 1) ^ 1, abort_flag, a.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            unsigned char* bst = smem + SU_OFF_B + st * SU_STAGE;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = r0 + 4 * i;
                const uint4 w = cur[i];
                const uint4 lo = make_uint4(su_px2<P>(w.x, 0), su_px2<P>(w.x, 1), su_px2<P>(w.y, 0), su_px2<P>(w.y, 1));
                const uint4 hi = make_uint4(su_px2<P>(w.z, 0), su_px2<P>(w.z, 1), su_px2<P>(w.w, 0), su_px2<P>(w.w, 1));
                *reinterpret_cast<uint4*>(bst + (2 * r) * (NT * 16) + nb * 16) = lo;
                *reinterpret_cast<uint4*>(bst + (2 * r + 1) * (NT * 16) + nb * 16) = hi;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_BF + 8 * st);
#pragma unroll
            for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
        }
    } else {
        // ---- epilogue warps: lane quarter q = warp % 4 (tensor-memory
        // access rule), column half ch; first they copy half 0 of the
        // operand table into tensor memory
        const int e = warp - W_EPI, q = warp & 3, ch = e >> 2;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        bool alive = true;
        {
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar + SU_TABF, 0, abort_flag, a.status);
            alive = __shfl_sync(0xffffffffu, ok, 0) != 0;
        }
        if (alive) {
            // part ch (0: hi, 1: lo) of half 0, staged at the region of half 1's part ch
            if (kSplit || ch == 0) {
                const uint32_t* tabs =
                    reinterpret_cast<const uint32_t*>(smem + (ch ? SU_OFF_A1LO : SU_OFF_A1HI)) + 32 * q + lane;
#pragma unroll 1
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = tabs[(cb * 32 + i) * 128];
                    tmem_st32(tmem + lane_base + ch * 128 + cb * 32, v);
                }
                tmem_wait_st();
            }
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_TABE);
        }
        griddep_wait();
        const float inv = 1.f / SU_SCALE;
        for (int j = 0; j < my_n && alive; ++j) {
            const int acc = j & 1, u = j >> 1, is = j % SU_I;
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait(bar + SU_ACCF + 8 * acc, u & 1, abort_flag, a.status);
                if (ok) ok = mbar_wait(bar + SU_INF + 8 * is, (j / SU_I) & 1, abort_flag, a.status);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc5_fence_after();
            const SuInfo& I = info[is];
            const int kmax = I.kmax;
            const int64_t base = I.base;
            const uint32_t my_pk = I.pk[32 * ch + lane];      // for the offsets below
            // the accumulator is read out first and released at once, so the
            // next tile's products overlap these stores
            const bool h0 = 32 * q < kmax, h1 = 128 + 32 * q < kmax;   // warp-uniform
            uint32_t v0[32], v1[32];
            const uint32_t ta = tmem + lane_base + 256 + 128 * acc + 32 * ch;
            if (h0) tmem_ld32(ta, v0);
            if (h1) tmem_ld32(ta + 64, v1);
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_ACCE + 8 * acc);
            // block i's (offset, count) comes from lane i by a shuffle, not a
            // shared-memory load, so nothing orders it after the stores
            float* const y = a.coeffs;
            if (h0) {
                const int rank = 32 * q + lane;
                const int64_t yb = base + rank;
                const int lim = (int)min(a.capacity - yb, (int64_t)1 << 30);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const uint32_t pk = __shfl_sync(0xffffffffu, my_pk, i);
                    const int m = (int)(pk >> 16), rel = (int)(pk & 0xFFFFu);
                    st_pred(y + yb + rel, __uint_as_float(v0[i]) * inv, rank < m && rel < lim);
                }
            }
            if (h1) {
                const int rank = 128 + 32 * q + lane;
                const int64_t yb = base + rank;
                const int lim = (int)min(a.capacity - yb, (int64_t)1 << 30);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const uint32_t pk = __shfl_sync(0xffffffffu, my_pk, i);
                    const int m = (int)(pk >> 16), rel = (int)(pk & 0xFFFFu);
                    st_pred(y + yb + rel, __uint_as_float(v1[i]) * inv, rank < m && rel < lim);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_INE + 8 * is);
            // global offsets of the tile's blocks (and the total after the last block)
            if (q == 0) {
                const int64_t b0 = tile_b0(j);
                const int i = 32 * ch + lane;
                if (b0 + i < ntot) {
                    const int64_t o = base + (int64_t)(my_pk & 0xFFFFu);
                    a.offsets[b0 + i] = o;
                    if (b0 + i == ntot - 1) {
                        a.offsets[ntot] = o + (int64_t)(my_pk >> 16);
                        if (o + (int64_t)(my_pk >> 16) > a.capacity) set_status(a.status, ABCS_DEV_CAPACITY);
                    }
                }
            }
        }
    }
    tc5_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc5_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int P>
cudaError_t launch_sense_umma_p(const SenseArgs& a, cudaStream_t s) {
    const int64_t ntot = (int64_t)a.g.n_img * a.g.n_blocks;
    if (ntot <= 0) return cudaSuccess;
    int dev, sms;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaFuncSetAttribute(sense_umma_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SU_SMEM);
    if (e) return e;
    const int64_t T = (ntot + NT - 1) / NT;
    const int grid = (int)(T < sms ? T : sms);
    return launch_pdl(sense_umma_kernel<P>, dim3(grid), dim3(SU_THREADS), SU_SMEM, s, a, ntot);
}

}  // namespace

cudaError_t setup_sense_umma() {
    sphi_setup_kernel<<<dim3(128, 2), 128>>>();
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaDeviceSynchronize();
    return e;
}

// The bulk copies of pixel rows need 16-byte aligned rows and images.
bool sense_umma_usable(const SenseArgs& a) {
    if (a.g.B != 16) return false;
    const uintptr_t al = reinterpret_cast<uintptr_t>(a.img) | (uintptr_t)a.g.pitch |
                         (uintptr_t)(a.g.n_img > 1 ? a.g.img_stride : 0);
    return (al & 15) == 0;
}

cudaError_t launch_sense_umma(const SenseArgs& a, cudaStream_t s) {
    switch (a.precision) {
        case kSP16: return launch_sense_umma_p<kSP16>(a, s);
        case kSPB16: return launch_sense_umma_p<kSPB16>(a, s);
        case kSPB1: return launch_sense_umma_p<kSPB1>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace abcs
