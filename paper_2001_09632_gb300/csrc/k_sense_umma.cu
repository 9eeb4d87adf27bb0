// Sensing on the 5th-generation tensor cores (B = 16): the measurements of
// a tile of 32 blocks as ONE GEMM against the zigzag-ordered DCT basis.
//
// With phi_k the basis image of zigzag rank k (phi_k[16 r + c] =
// D[u_k][r] D[v_k][c], Eq. 1 and the zigzag order of Sec. IV), block b's
// rank-k measurement (a row of Eq. 26's A applied to the block) is
//   y_b[k] = sum_p phi_k[p] x_b[p].
// For a tile of NT = 32 blocks and the ranks of one half h (k = 128 h + m):
//   Y_h[m][n] = sum_p 16 phi_{128 h + m}[p] x_n[p] / 16
//   (M = 128 ranks, N = 32 blocks, K = 256 pixels)
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
//   [256, 384)  A of half 1, hi words (ranks 128 .. 255)
//   [384, 512)  two accumulators of 64 columns: half 0 (32 blocks) then half 1
// The lo words of half 1 are the shared-memory A operand of its second
// product.  Half 1 is computed only for tiles whose largest count exceeds
// 128 (most tiles stop at rank 127 at subrates up to 0.3).
//
// Roles (10 warps, one CTA per SM, tiles c, c + G, c + 2G, ...):
//   warp 0      tensor-memory allocation; lane 0 loads the operand table
//               and issues the MMAs
//   warp 1      producer: pixel rows of a tile into a ring of raw slots by
//               bulk copies (one per pixel row of each run of consecutive
//               blocks in a block row); after the wait for the pilot kernel,
//               each tile's counts, global offsets and largest count
//   warps 2-5   converters: raw bytes -> FP16 / BF16 K-major B operand
//               (lane = block, warp = pixel rows), one 16-byte store per
//               8 pixels, no bank conflicts
//   warps 6-9   epilogue: warp w reads lanes 32 (w % 4) .. (32 ranks) of
//               the tile's 32 columns (blocks) and stores rank k of block n
//               to y[offset_n + k] when k < m_n (a warp store covers 32
//               consecutive coefficients of one block); it also writes the
//               global offsets
// The pixel staging and the half-0 products of the first tiles need no
// allocation result, so they run while the pilot kernel finishes (PDL).
// Every wait is bounded: on expiry ABCS_DEV_TIMEOUT is set and an abort flag
// ends every role; copies and MMAs in flight are drained before the CTA
// frees its tensor memory.
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

constexpr int NT = 32;                 // blocks per tile (the MMA's N)
constexpr int SU_R = 4;                // raw pixel slots
constexpr int SU_S = 3;                // B operand stages
constexpr int SU_I = 4;                // metadata slots
constexpr float SU_SCALE = 16.f;
constexpr uint32_t SU_PART = 65536;    // bytes of one operand-table part
constexpr uint32_t SU_STAGE = NT * 512;   // 32 K chunks of NT rows x 16 bytes
constexpr uint32_t SU_RAW = NT * 256;     // 16 pixel rows of NT blocks x 16 bytes

struct SuInfo {
    int64_t off[NT];   // global offset of the block's first coefficient
    int m[NT];         // the block's count (0 past the batch or when flagged)
    int kmax;          // largest count of the tile
    int pad;
};

constexpr uint32_t SU_OFF_A1LO = 0;                               // also staging of the table parts
constexpr uint32_t SU_OFF_B = SU_OFF_A1LO + SU_PART;
constexpr uint32_t SU_OFF_RAW = SU_OFF_B + SU_S * SU_STAGE;
constexpr uint32_t SU_OFF_INFO = SU_OFF_RAW + SU_R * SU_RAW;
constexpr uint32_t SU_OFF_BAR = SU_OFF_INFO + SU_I * sizeof(SuInfo);
// mbarriers
constexpr uint32_t SU_RAWF = 0, SU_RAWE = SU_RAWF + 8 * SU_R, SU_BF = SU_RAWE + 8 * SU_R, SU_BE = SU_BF + 8 * SU_S,
                   SU_ACCF = SU_BE + 8 * SU_S, SU_ACCE = SU_ACCF + 16, SU_INF = SU_ACCE + 16,
                   SU_INE = SU_INF + 8 * SU_I, SU_TABF = SU_INE + 8 * SU_I, SU_TABE = SU_TABF + 8,
                   SU_DRAIN = SU_TABE + 8, SU_NBAR = SU_DRAIN + 8;
constexpr uint32_t SU_OFF_MISC = SU_OFF_BAR + SU_NBAR;            // tensor-memory address, abort flag
constexpr size_t SU_SMEM = SU_OFF_MISC + 16;
constexpr int SU_THREADS = 10 * 32;
static_assert(SU_OFF_B % 1024 == 0 && SU_OFF_RAW % 16 == 0 && SU_OFF_INFO % 16 == 0 && SU_OFF_BAR % 8 == 0,
              "shared layout");
static_assert(SU_SMEM <= 232448, "shared memory of the tensor-memory sensing kernel");

// Operand table per precision, four 64 KB parts of 16 phi (rows = ranks of
// a half, K = pixels):
//   parts 0, 1, 2: tensor-memory words of half 0 hi, half 0 lo, half 1 hi,
//                  word [c][m] = (A[m][2c], A[m][2c + 1])
//   part 3:        half 1 lo as its shared-memory K-major image,
//                  byte 2048 kc + 16 m + 2 e = A[m][8 kc + e]
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
        t[2][c * 128 + m] = hi;
        // pixels 2c, 2c + 1: chunk kc = 2c / 8, word (2c % 8) / 2 of row m
        t[3][(c >> 2) * 512 + m * 4 + (c & 3)] = lo;
    }
}

__global__ void sphi_setup_kernel() {     // grid (128 columns, 2 halves), block 128 (ranks)
    const int c = blockIdx.x, half = blockIdx.y, m = threadIdx.x;
    sphi_setup_p<kSP16>(half, m, c);
    sphi_setup_p<kSPB16>(half, m, c);
    sphi_setup_p<kSPB1>(half, m, c);
}

// D (tensor memory) (+)= A (shared-memory descriptor) * B (shared-memory descriptor)
ABCS_D void umma_smem_a(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
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

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (t == 32) {
        for (int i = 0; i < SU_R; ++i) {
            mbar_init(bar + SU_RAWF + 8 * i, 1);
            mbar_init(bar + SU_RAWE + 8 * i, 4);
        }
        for (int i = 0; i < SU_S; ++i) {
            mbar_init(bar + SU_BF + 8 * i, 4);
            mbar_init(bar + SU_BE + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar + SU_ACCF + 8 * i, 1);
            mbar_init(bar + SU_ACCE + 8 * i, 4);
        }
        for (int i = 0; i < SU_I; ++i) {
            mbar_init(bar + SU_INF + 8 * i, 1);
            mbar_init(bar + SU_INE + 8 * i, 4);
        }
        mbar_init(bar + SU_TABF, 1);
        mbar_init(bar + SU_TABE, 4);
        mbar_init(bar + SU_DRAIN, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort_flag = 0;
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- operand table, then the MMA issuer
        if (lane == 0) {
            const uint32_t* tab = &g_sphi[su_pidx<P>()][0][0];
            bool alive = true;
            // parts 0 .. 2 staged in the A1lo region and copied into tensor
            // memory by the epilogue warps; part 3 lands there last
            int ph = 0;
            for (int part = 0; part < 4 && alive; ++part) {
                if (!kSplit && (part == 1 || part == 3)) continue;
                mbar_arrive_tx(bar + SU_TABF, SU_PART);
                bulk_g2s(sb + SU_OFF_A1LO, tab + part * (SU_PART / 4), SU_PART, bar + SU_TABF);
                if (!mbar_wait(bar + SU_TABF, ph & 1, abort_flag, a.status)) alive = false;
                if (part != 3 && alive) {
                    // the epilogue warps have copied this part into tensor memory
                    if (!mbar_wait(bar + SU_TABE, ph & 1, abort_flag, a.status)) alive = false;
                }
                ++ph;
            }
            tc5_fence_after();
            for (int j = 0; j < my_n && alive; ++j) {
                const int acc = j & 1, st = j % SU_S, is = j % SU_I;
                if (!mbar_wait(bar + SU_ACCE + 8 * acc, ((j >> 1) & 1) ^ 1, abort_flag, a.status)) break;
                if (!mbar_wait(bar + SU_BF + 8 * st, (j / SU_S) & 1, abort_flag, a.status)) break;
                tc5_fence_after();
                const uint32_t d0 = tmem + 384 + 64 * acc, d1 = d0 + 32;
                const uint32_t bst = sb + SU_OFF_B + st * SU_STAGE;
#pragma unroll 4
                for (int ks = 0; ks < 16; ++ks) {
                    const uint64_t bd = umma_desc(bst + ks * 1024, 512, 128);
                    umma_tmem_a(d0, tmem + 8 * ks, bd, IDESC, ks > 0 ? 1u : 0u);
                    if constexpr (kSplit) umma_tmem_a(d0, tmem + 128 + 8 * ks, bd, IDESC, 1u);
                }
                // half 1 only where some block of the tile needs ranks >= 128
                if (!mbar_wait(bar + SU_INF + 8 * is, (j / SU_I) & 1, abort_flag, a.status)) break;
                if (info[is].kmax > 128) {
#pragma unroll 4
                    for (int ks = 0; ks < 16; ++ks) {
                        const uint64_t bd = umma_desc(bst + ks * 1024, 512, 128);
                        umma_tmem_a(d1, tmem + 256 + 8 * ks, bd, IDESC, ks > 0 ? 1u : 0u);
                        if constexpr (kSplit)
                            umma_smem_a(d1, umma_desc(sb + SU_OFF_A1LO + ks * 4096, 2048, 128), bd, IDESC, 1u);
                    }
                }
                umma_commit(bar + SU_BE + 8 * st);        // the stage is free once these complete
                umma_commit(bar + SU_ACCF + 8 * acc);     // the tile's accumulators are ready
            }
            umma_commit(bar + SU_DRAIN);
            mbar_drain(bar + SU_DRAIN, 0, a.status);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- producer
        const uint8_t* img = a.img;
        auto pixels = [&](int j) -> bool {
            const int slot = j % SU_R;
            if (j >= SU_R) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(bar + SU_RAWE + 8 * slot, ((j / SU_R) & 1) ^ 1, abort_flag, a.status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
            }
            const int64_t b0 = ((int64_t)blockIdx.x + (int64_t)j * G) * NT;
            const int n = (int)(ntot - b0 < NT ? ntot - b0 : NT);
            // lane = block of the tile; a run starts at the tile's first block
            // and at every block-row start
            int k = 0, bi = 0, bj = 0;
            if (lane < n) su_coords(g, b0 + lane, k, bi, bj);
            const bool start = lane < n && (lane == 0 || bj == 0);
            const int len = start ? min(n - lane, g.nbw - bj) : 0;
            if (lane == 0) mbar_arrive_tx(bar + SU_RAWF + 8 * slot, (uint32_t)n * 256u);
            __syncwarp();
            if (start) {
                const uint8_t* src = img + (int64_t)k * g.img_stride + (int64_t)(bi * 16) * g.pitch + bj * 16;
                const uint32_t dst = sb + SU_OFF_RAW + slot * SU_RAW + lane * 16;
                for (int r = 0; r < 16; ++r)
                    bulk_g2s(dst + r * (NT * 16), src + (int64_t)r * g.pitch, (uint32_t)len * 16u,
                             bar + SU_RAWF + 8 * slot);
            }
            return true;
        };
        auto meta = [&](int j) -> bool {
            const int is = j % SU_I;
            if (j >= SU_I) {
                int ok = 1;
                if (lane == 0) ok = mbar_wait(bar + SU_INE + 8 * is, ((j / SU_I) & 1) ^ 1, abort_flag, a.status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
            }
            const int64_t b0 = ((int64_t)blockIdx.x + (int64_t)j * G) * NT;
            const int n = (int)(ntot - b0 < NT ? ntot - b0 : NT);
            int m = 0;
            int64_t off = 0;
            bool bad = false;
            if (lane < n) {
                int k, bi, bj;
                su_coords(g, b0 + lane, k, bi, bj);
                m = __ldg(a.counts + b0 + lane);
                off = __ldg(a.offsets + b0 + lane) + __ldg(a.img_base + k);
                if (m < 0 || m > 256 || off < 0) {
                    bad = true;
                    m = 0;
                    off = 0;
                }
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(a.status, ABCS_DEV_BADCOUNT);
            SuInfo& I = info[is];
            I.m[lane] = m;
            I.off[lane] = off;
            int km = m;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
            if (lane == 0) I.kmax = km;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_INF + 8 * is);
            return true;
        };
        // the first slots' pixels do not depend on the allocation: they are
        // copied before the wait for the pilot kernel (which lets this grid
        // start once that kernel has passed its own wait)
        int jp = 0;
        bool ok = true;
        for (; jp < SU_R && jp < my_n && ok; ++jp) ok = pixels(jp);
        griddep_wait();
        for (int j = 0; j < my_n && ok; ++j) {
            ok = meta(j);
            if (ok && jp < my_n) ok = pixels(jp++);
        }
        // copies still in flight land before the CTA leaves
        if (lane == 0)
            for (int jj = jp > SU_R ? jp - SU_R : 0; jj < jp; ++jj)
                mbar_drain(bar + SU_RAWF + 8 * (jj % SU_R), (jj / SU_R) & 1, a.status);
    } else if (warp < 6) {
        // ---- converters: warp wl = warp - 2 takes pixel rows wl, wl + 4, wl + 8, wl + 12 of
        // every block (lane = block)
        const int wl = warp - 2;
        for (int j = 0; j < my_n; ++j) {
            const int slot = j % SU_R, st = j % SU_S;
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait(bar + SU_RAWF + 8 * slot, (j / SU_R) & 1, abort_flag, a.status);
                if (ok) ok = mbar_wait(bar + SU_BE + 8 * st, ((j / SU_S) & 1) ^ 1, abort_flag, a.status);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const unsigned char* raw = smem + SU_OFF_RAW + slot * SU_RAW;
            unsigned char* bst = smem + SU_OFF_B + st * SU_STAGE;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wl + 4 * i;
                const uint4 w = *reinterpret_cast<const uint4*>(raw + r * (NT * 16) + lane * 16);
                const uint4 lo = make_uint4(su_px2<P>(w.x, 0), su_px2<P>(w.x, 1), su_px2<P>(w.y, 0), su_px2<P>(w.y, 1));
                const uint4 hi = make_uint4(su_px2<P>(w.z, 0), su_px2<P>(w.z, 1), su_px2<P>(w.w, 0), su_px2<P>(w.w, 1));
                *reinterpret_cast<uint4*>(bst + (2 * r) * (NT * 16) + lane * 16) = lo;
                *reinterpret_cast<uint4*>(bst + (2 * r + 1) * (NT * 16) + lane * 16) = hi;
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar + SU_BF + 8 * st);
                mbar_arrive(bar + SU_RAWE + 8 * slot);
            }
        }
    } else {
        // ---- epilogue warps; first they copy the operand table into tensor memory
        const int q = warp & 3;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        bool alive = true;
        int ph = 0;
        for (int part = 0; part < 3 && alive; ++part) {
            if (!kSplit && part == 1) continue;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar + SU_TABF, ph & 1, abort_flag, a.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) {
                alive = false;
                break;
            }
            const uint32_t* tabs = reinterpret_cast<const uint32_t*>(smem + SU_OFF_A1LO) + 32 * q + lane;
#pragma unroll 1
            for (int cb = 0; cb < 4; ++cb) {
                uint32_t v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = tabs[(cb * 32 + i) * 128];
                tmem_st32(tmem + lane_base + part * 128 + cb * 32, v);
            }
            tmem_wait_st();
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + SU_TABE);
            ++ph;
        }
        griddep_wait();
        const float inv = 1.f / SU_SCALE;
        for (int j = 0; j < my_n && alive; ++j) {
            const int acc = j & 1, is = j % SU_I;
            int ok = 1;
            if (lane == 0) {
                ok = mbar_wait(bar + SU_ACCF + 8 * acc, (j >> 1) & 1, abort_flag, a.status);
                if (ok) ok = mbar_wait(bar + SU_INF + 8 * is, (j / SU_I) & 1, abort_flag, a.status);
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc5_fence_after();
            const SuInfo& I = info[is];
            const int kmax = I.kmax;
            const int64_t b0 = ((int64_t)blockIdx.x + (int64_t)j * G) * NT;
            const int n = (int)(ntot - b0 < NT ? ntot - b0 : NT);
            for (int h = 0; h < 2; ++h) {
                const int k0 = 128 * h + 32 * q;      // this warp's first rank
                if (k0 >= kmax) continue;             // warp-uniform: no block needs these ranks
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + 384 + 64 * acc + 32 * h, v);
                const int rank = k0 + lane;
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const int m = I.m[i];
                    if (k0 >= m) continue;            // warp-uniform
                    const int64_t o = I.off[i] + rank;
                    if (rank < m) {
                        if (o < a.capacity) a.coeffs[o] = __uint_as_float(v[i]) * inv;
                        else set_status(a.status, ABCS_DEV_CAPACITY);
                    }
                }
            }
            // global offsets of the tile's blocks
            if (q == 0 && lane < n) {
                a.offsets[b0 + lane] = I.off[lane];
                if (b0 + lane == ntot - 1) a.offsets[ntot] = I.off[lane] + I.m[lane];
            }
            tc5_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar + SU_ACCE + 8 * acc);
                mbar_arrive(bar + SU_INE + 8 * is);
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
