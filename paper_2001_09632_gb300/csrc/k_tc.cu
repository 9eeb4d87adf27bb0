// Tensor-core block DCT for B = 16: sensing and reconstruction as chains of
// 16x16 matrix products on mma.sync.m16n8k16 with FP32 accumulation.
//
// One warp owns one 16x16 block at a time and keeps it in MMA fragments
// through both transform stages (the accumulator layout of the first
// product is the A-operand layout of the second), so no shared-memory
// transpose is needed.  Persistent CTAs walk equal contiguous block ranges
// in 32-block segments whose input is staged with cp.async while the
// previous segment is transformed.
//
// The file also holds recon_umma_kernel, the reconstruction as one tcgen05
// GEMM per 128-block tile against the DCT basis images kept in tensor
// memory (selected with ABCS_RECON_TC=umma; slower than the per-block
// kernel on the measured workloads).
//
// Precisions (abcs_precision):
//   TC_FP16X2  operands split v = hi + lo in FP16; products hi*hi + lo*hi + hi*lo
//   TC_BF16X2  the same split in BF16
//   TC_BF16    single BF16 product hi*hi
// Pixels are integers <= 255, exact in FP16 and BF16, so the sensing input
// needs no split.
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "abcs_common.cuh"
#include "umma.cuh"

namespace abcs {
ABCS_TU_TABLES(tc)
}  // namespace abcs

#include "alloc_dev.cuh"
#include "dct_tile.cuh"
#include "dd_exact.cuh"
#include "tc_frag.cuh"

namespace abcs {

namespace {

// Operand fragments of the constant factors D and D^T (hi and lo words), per
// precision, fragment set and lane.  They are split from the FP64 table once
// per device by tc_frag_setup_kernel: doing it in every CTA's prologue kept
// the narrow FP64 pipe of this GPU busy for a large part of each launch.
enum { kSetSenseA = 0, kSetSenseB = 1, kSetReconA = 2, kSetReconB = 3 };
__device__ uint32_t g_tc_frag[3][4][8][32];

// A fragment of the sensing row transform: A[m][k] = D[m][pi(k)] with
// pi(2q + e) = 4q + e, pi(2q + 8 + e) = 4q + 2 + e (e = 0, 1).
template <int P>
ABCS_D void load_a_perm(uint32_t (&h)[4], uint32_t (&l)[4]) {
    const Frag f;
    split2d<P>(Dd<16>(f.g, 4 * f.q), Dd<16>(f.g, 4 * f.q + 1), h[0], l[0]);
    split2d<P>(Dd<16>(f.g + 8, 4 * f.q), Dd<16>(f.g + 8, 4 * f.q + 1), h[1], l[1]);
    split2d<P>(Dd<16>(f.g, 4 * f.q + 2), Dd<16>(f.g, 4 * f.q + 3), h[2], l[2]);
    split2d<P>(Dd<16>(f.g + 8, 4 * f.q + 2), Dd<16>(f.g + 8, 4 * f.q + 3), h[3], l[3]);
}

template <int P>
ABCS_D void frag_setup_p() {
    const int lane = threadIdx.x & 31;
    uint32_t (*t)[8][32] = g_tc_frag[pidx<P>()];
    uint32_t h[4], l[4], bh[2][2], bl[2][2];
    auto put_a = [&](int set) {
        for (int i = 0; i < 4; ++i) {
            t[set][i][lane] = h[i];
            t[set][4 + i][lane] = l[i];
        }
    };
    auto put_b = [&](int set) {
        for (int i = 0; i < 4; ++i) {
            t[set][i][lane] = bh[i >> 1][i & 1];
            t[set][4 + i][lane] = bl[i >> 1][i & 1];
        }
    };
    load_a_perm<P>(h, l);
    put_a(kSetSenseA);
    load_b_const<P>(true, bh, bl);
    put_b(kSetSenseB);
    load_a_const<P>(true, h, l);
    put_a(kSetReconA);
    load_b_const<P>(false, bh, bl);
    put_b(kSetReconB);
}

__global__ void tc_frag_setup_kernel() {
    frag_setup_p<kP16>();
    frag_setup_p<kPB16>();
    frag_setup_p<kPB1>();
}

template <int P>
ABCS_D void frag_a(int set, uint32_t (&h)[4], uint32_t (&l)[4]) {
    const uint32_t* t = &g_tc_frag[pidx<P>()][set][0][threadIdx.x & 31];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = t[32 * i];
        l[i] = t[32 * (4 + i)];
    }
}

template <int P>
ABCS_D void frag_b(int set, uint32_t (&h)[2][2], uint32_t (&l)[2][2]) {
    const uint32_t* t = &g_tc_frag[pidx<P>()][set][0][threadIdx.x & 31];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i >> 1][i & 1] = t[32 * i];
        l[i >> 1][i & 1] = t[32 * (4 + i)];
    }
}

// ---------------------------------------------------------------------------
// Segments.  The batch's blocks (raster order within an image, images
// consecutive) are split into one contiguous range per CTA, equal to within
// one block, so every CTA has the same work.  A CTA walks its range in
// segments of SEG = RSEG = 32 blocks (a segment may cross block rows and
// images):
// their packed coefficients form one contiguous range, moved between global
// and shared memory with coalesced 16-byte copies; the next segment's input
// is copied (cp.async) while the current one is transformed, and each warp
// transforms four blocks of the segment.
// ---------------------------------------------------------------------------
#ifndef ABCS_RECON_RSEG
#define ABCS_RECON_RSEG 32
#endif
#ifndef ABCS_RECON_DEPTH
#define ABCS_RECON_DEPTH 1
#endif
#ifndef ABCS_SENSE_DEPTH
#define ABCS_SENSE_DEPTH 1
#endif
constexpr int SEG = 32;                        // sensing segment (blocks)
constexpr int SDEPTH = ABCS_SENSE_DEPTH;       // sensing segments staged ahead
constexpr int SNB = SDEPTH + 1, SNM = SDEPTH + 2;   // pixel buffers, metadata slots
constexpr int RSEG = ABCS_RECON_RSEG;          // reconstruction segment (blocks)
constexpr int RDEPTH = ABCS_RECON_DEPTH;       // reconstruction segments staged ahead
constexpr int RNB = RDEPTH + 1, RNM = RDEPTH + 2;   // stage buffers, metadata slots
template <int S>
constexpr int seg_floats() { return S * 256 + 4; }   // packed range of a segment + alignment shift
constexpr int kSegFloats = seg_floats<SEG>();
constexpr int kRSegFloats = seg_floats<RSEG>();

struct SegGeom {
    int64_t b0;        // first block of the segment (index over the batch)
    int nblk;
};

// the CTA's block range [r0, r1) and its segment j
ABCS_D void cta_range(int64_t ntot, int64_t* r0, int64_t* r1) {
    *r0 = ntot * blockIdx.x / gridDim.x;
    *r1 = ntot * (blockIdx.x + 1) / gridDim.x;
}

template <int S>
ABCS_D SegGeom seg_geom(int64_t r0, int64_t r1, int j) {
    SegGeom r;
    r.b0 = r0 + (int64_t)j * S;
    r.nblk = (int)min((int64_t)S, r1 - r.b0);
    return r;
}

template <int SEG>
struct SegMeta {
    int64_t start;     // index of the segment's first coefficient in the packed vector
    int n;             // coefficients of the segment
    int sh;            // start & 3: stage position of coefficient `start`
    int rel[SEG];      // block offsets relative to start
    int cnt[SEG];      // block counts
    int64_t pos[SEG];  // block's top-left pixel: recon, in the output; sense, byte offset in the input
    SegGeom sg;
};

ABCS_D int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block b of the batch -> image k, block row bi, block column bj (b < 2^31)
ABCS_D void block_coords(const ImgGeom& g, int64_t b, int& k, int& bi, int& bj) {
    const int bb = (int)b, nB = (int)g.n_blocks;
    k = bb / nB;
    const int i = bb - k * nB;
    bi = i / g.nbw;
    bj = i - bi * g.nbw;
}

// Metadata of a segment as loaded by warp 0 (lane = block of the segment).
// Loads are issued two segments ahead and written to shared memory one
// segment ahead, so their latency is hidden behind a segment's transforms.
struct MetaRaw {
    int64_t off;       // the block's offset (recon: global; sense: image-local + image base)
    int64_t pos;       // the block's pixel position
    int m;             // the block's count
};

ABCS_D MetaRaw recon_meta_load(const ReconArgs& a, const SegGeom& sg) {
    const int lane = threadIdx.x & 31;
    MetaRaw r;
    r.off = 0;
    r.pos = 0;
    r.m = 0;
    if (lane < sg.nblk) {
        const int64_t b = sg.b0 + lane;
        r.off = __ldg(a.offsets + b);
        r.m = __ldg(a.counts + b);
        int k, bi, bj;
        block_coords(a.g, b, k, bi, bj);
        r.pos = (int64_t)k * a.g.Hc * a.g.Wc + (int64_t)(bi * 16) * a.g.Wc + bj * 16;
    }
    return r;
}

// Inconsistent counts or offsets are flagged and the block is treated as
// unmeasured, so every stage access stays inside the segment's buffer.
ABCS_D void recon_meta_store(const ReconArgs& a, const SegGeom& sg, const MetaRaw& r, SegMeta<RSEG>& M) {
    const int lane = threadIdx.x & 31;
    int64_t off = r.off;
    int m = r.m;
    int64_t start = __shfl_sync(0xffffffffu, off, 0);
    bool bad = false;
    if (start < 0) {
        bad = true;
        start = 0;
        off = 0;
        m = 0;
    }
    int64_t rel = off - start;
    if (lane < sg.nblk) {
        if (m < 0 || m > 256) { bad = true; m = m < 0 ? 0 : 256; }
        if (rel < 0 || rel + m > RSEG * 256) { bad = true; rel = 0; m = 0; }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(a.status, ABCS_DEV_BADCOUNT);
    const int end = warp_max(lane < sg.nblk ? (int)(rel + m) : 0);
    if (lane < RSEG) {
        M.rel[lane] = (int)rel;
        M.cnt[lane] = m;
        M.pos[lane] = r.pos;
    }
    if (lane == 0) {
        M.start = start;
        M.n = end;
        M.sh = (int)(start & 3);
        M.sg = sg;
    }
}

// ---------------------------------------------------------------------------
// reconstruct: X = D^T C D.  Stage 1 Y = D^T C (A = D^T constant, B = C
// gathered by zigzag rank from the staged segment); stage 2 X = Y D (A = Y
// straight from stage 1's accumulators, B = D constant).
// ---------------------------------------------------------------------------
constexpr size_t kReconSmem = RNB * kRSegFloats * sizeof(float) + RNM * sizeof(SegMeta<RSEG>);
constexpr size_t kSenseSmem = SNB * 16 * SEG * 16 + kSegFloats * sizeof(float) + SNM * sizeof(SegMeta<SEG>);

template <int P>
__global__ void __launch_bounds__(256, 3) recon_tc_kernel(ReconArgs a, int64_t ntot) {
    extern __shared__ __align__(16) unsigned char smem[];
    float (*stage)[kRSegFloats] = reinterpret_cast<float (*)[kRSegFloats]>(smem);
    SegMeta<RSEG>* meta = reinterpret_cast<SegMeta<RSEG>*>(smem + RNB * kRSegFloats * sizeof(float));
    const int warp = threadIdx.x >> 5;
    const Frag f;
    uint32_t ATh[4], ATl[4], DBh[2][2], DBl[2][2];
    frag_a<P>(kSetReconA, ATh, ATl);
    frag_b<P>(kSetReconB, DBh, DBl);
    // 4 x the ranks of the 8 coefficients this lane feeds into B = C: (2q + e, g + 8 nt), e in {0,1,8,9}
    // (byte offsets in the staged segment)
    int rkb[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rkb[nt][i] = 4 * zz_rank(2 * f.q + (i & 1) + 8 * (i >> 1), f.g + 8 * nt, 16);

    griddep_wait();
    const ImgGeom& g = a.g;
    int64_t r0, r1;
    cta_range(ntot, &r0, &r1);
    const int nseg = (int)((r1 - r0 + RSEG - 1) / RSEG);
    if (nseg <= 0) return;
    const int lo = f.g * g.Wc + 2 * f.q;
    // segments j + 1 .. j + RDEPTH are in flight while segment j is
    // transformed: RDEPTH + 1 stage buffers, RDEPTH + 2 metadata slots (warp 0
    // stores segment j + RDEPTH's metadata while the other warps may still
    // read segment j - 1's), metadata loads one segment further ahead
    MetaRaw raw;
    if (warp == 0) {
        for (int d = 0; d < RDEPTH && d < nseg; ++d)
            recon_meta_store(a, seg_geom<RSEG>(r0, r1, d), recon_meta_load(a, seg_geom<RSEG>(r0, r1, d)), meta[d]);
        if (RDEPTH < nseg) raw = recon_meta_load(a, seg_geom<RSEG>(r0, r1, RDEPTH));
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < RDEPTH; ++d) {
        if (d < nseg) stage_in_async(stage[d], a.coeffs, meta[d].start, meta[d].n);
        cp_async_commit();
    }
    int mi = 0, bi = 0;                         // metadata slot (j mod RNM) and stage buffer (j mod RNB) of segment j
    int mn = RDEPTH % RNM, bn = RDEPTH % RNB;   // the same for segment j + RDEPTH
    for (int j = 0; j < nseg; ++j) {
        const int jn = j + RDEPTH;
        if (jn < nseg && warp == 0) {
            recon_meta_store(a, seg_geom<RSEG>(r0, r1, jn), raw, meta[mn]);
            if (jn + 1 < nseg) raw = recon_meta_load(a, seg_geom<RSEG>(r0, r1, jn + 1));
        }
        cp_async_wait_group<RDEPTH - 1>();      // this thread's copies of segment j have landed
        __syncthreads();
        if (jn < nseg) stage_in_async(stage[bn], a.coeffs, meta[mn].start, meta[mn].n);
        cp_async_commit();

        const SegMeta<RSEG>& M = meta[mi];
        const SegGeom sg = M.sg;
        const uint32_t st = smem_u32(stage[bi] + M.sh);
#pragma unroll
        for (int c = warp; c < sg.nblk; c += 8) {
            const int m4 = 4 * M.cnt[c];
            const uint32_t sb = st + 4u * (uint32_t)M.rel[c];
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float cv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) cv[i] = lds_f_lt(sb + (uint32_t)rkb[nt][i], rkb[nt][i], m4);
                split2<P>(cv[0], cv[1], bh[nt][0], bl[nt][0]);
                split2<P>(cv[2], cv[3], bh[nt][1], bl[nt][1]);
            }
            float Y[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
                mma_split<P>(Y[nt], ATh, ATl, bh[nt][0], bh[nt][1], bl[nt][0], bl[nt][1]);
            uint32_t Ah[4], Al[4];
            split2<P>(Y[0][0], Y[0][1], Ah[0], Al[0]);
            split2<P>(Y[0][2], Y[0][3], Ah[1], Al[1]);
            split2<P>(Y[1][0], Y[1][1], Ah[2], Al[2]);
            split2<P>(Y[1][2], Y[1][3], Ah[3], Al[3]);
            float X[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
                mma_split<P>(X[nt], Ah, Al, DBh[nt][0], DBh[nt][1], DBl[nt][0], DBl[nt][1]);

            const int64_t o = M.pos[c] + lo;
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
        }
        mi = mi + 1 == RNM ? 0 : mi + 1;
        bi = bi + 1 == RNB ? 0 : bi + 1;
        mn = mn + 1 == RNM ? 0 : mn + 1;
        bn = bn + 1 == RNB ? 0 : bn + 1;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// reconstruct on the 5th-generation tensor cores (the alternative to
// recon_tc_kernel, selected with ABCS_RECON_TC=umma).  With phi_k the DCT
// basis image of zigzag rank k (phi_k[16 r + c] = D[u_k][r] D[v_k][c]),
// block b's pixels are x_b = sum_{k < m_b} y_b[k] phi_k (the inverse of
// Eq. 1 with the unmeasured coefficients zero).  For a tile of KR_BLK blocks
// and pixel half h this is one GEMM,
//   X_h[p][i] = sum_k 16 phi_k[128 h + p] * y_i[k]     (M = 128 pixels, N = KR_BLK blocks, K = rank)
// A = 16 Phi_h (hi + lo words) stays in tensor memory for the whole launch
// (column k/2 of lane p holds ranks k, k + 1), B = the tile's coefficients
// (hi + lo) goes through shared memory in K stages of KR_KS ranks, and the
// FP32 accumulators are in tensor memory.  K stops at the tile's largest
// count, so the MMA work follows the measurements.  The three split products
// A_hi B_hi + A_lo B_hi + A_hi B_lo restore FP32 accuracy (one product for
// plain BF16); the factor 16 keeps the low words of Phi out of the FP16
// subnormal range and is divided out exactly in the epilogue.
// One CTA per SM; CTA c computes pixel half c & 1 of tiles c/2, c/2 + G/2, ...
//   warp 0      tensor-memory allocation; lane 0 issues the MMAs
//   warp 1      loader: the tile's packed coefficients (one contiguous range)
//               by one bulk copy into a ring of spans (up to 8 tiles in
//               flight); per-block offsets and counts, loaded a tile ahead,
//               and the tile's stage count
//   warps 2-9   converters: thread (block i, part) splits its share of the
//               stage's ranks into hi + lo and writes them K-major (no
//               swizzle) into the stage buffers
//   warps 10-13 epilogue (and, first, the tensor-memory copy of A from the
//               table staged by one bulk copy): warp w reads lanes
//               32 (w % 4) .. (its pixels) of the tile's columns (blocks);
//               each store of a warp covers two pixel rows of one block
// Every wait is bounded (ABCS_DEV_TIMEOUT and an abort flag that ends every
// role); copies and MMAs in flight are drained before the CTA frees its
// tensor memory and leaves.
// Measured on 64 x 512^2 (BBV r 0.3, FP16x2): 36 us against 23 us for
// recon_tc_kernel.  The MMAs keep the tensor pipe busy only ~14% of the
// time; each K stage costs a hand-off between eight converter warps and the
// MMA thread that the per-block mma.sync kernel does not pay, and both pixel
// halves convert the same coefficients, padded to the tile's largest count.
// ---------------------------------------------------------------------------
#ifndef ABCS_KR_BLK
#define ABCS_KR_BLK 128
#endif
#ifndef ABCS_KR_KS
#define ABCS_KR_KS 64
#endif
#ifndef ABCS_KR_NB
#define ABCS_KR_NB 2
#endif
constexpr int KR_BLK = ABCS_KR_BLK;                 // blocks per tile (the MMA's N: 64 or 128)
constexpr int KR_KS = ABCS_KR_KS;                   // ranks per K stage (32 or 64)
constexpr int KR_NB = ABCS_KR_NB;                   // stage buffers (a power of 2)
constexpr int KR_CH = KR_KS / 8;                    // 8-rank chunks per stage
constexpr int KR_TPB = 256 / KR_BLK;                // converter threads per block
constexpr int KR_CPT = KR_CH / KR_TPB;              // chunks per converter thread and stage
constexpr int KR_NACC = 256 / KR_BLK;               // accumulators (256 tensor-memory columns)
constexpr int KR_NSLOT = 8;                         // tiles in flight between loader and converters
constexpr int KR_RING = KR_BLK == 64 ? 2 * (KR_BLK * 256 + 8) : KR_BLK * 256 + 8;   // floats of the ring
constexpr uint32_t KR_CHUNK = KR_BLK * 16;          // one 8-rank chunk of all the tile's blocks
constexpr uint32_t KR_STAGE = 2 * KR_CH * KR_CHUNK; // hi chunks, then lo chunks
static_assert(KR_CPT >= 1 && KR_CH % KR_TPB == 0 && (KR_NB & (KR_NB - 1)) == 0, "stage geometry");
constexpr float KR_SCALE = 16.f;
struct KrInfo {
    int rel[KR_BLK];   // ring index of the block's first coefficient
    int m[KR_BLK];     // the block's count (0 for rows past the batch or flagged)
    int nst;           // K stages of the tile
    int pad[3];
};
constexpr uint32_t KR_OFF_STAGE = 0;
constexpr uint32_t KR_OFF_RAW = KR_NB * KR_STAGE;
constexpr uint32_t KR_OFF_INFO = KR_OFF_RAW + KR_RING * 4;
constexpr uint32_t KR_OFF_BAR = KR_OFF_INFO + KR_NSLOT * sizeof(KrInfo);
// mbarriers: ring full/empty per slot, stage full/empty per buffer, acc full/empty, drain
constexpr uint32_t KR_RAWF = 0, KR_RAWE = 8 * KR_NSLOT, KR_BF = 16 * KR_NSLOT, KR_BE = KR_BF + 8 * KR_NB,
                   KR_ACCF = KR_BE + 8 * KR_NB, KR_ACCE = KR_ACCF + 8 * KR_NACC, KR_DRAIN = KR_ACCE + 8 * KR_NACC,
                   KR_TAB = KR_DRAIN + 8;
constexpr uint32_t KR_OFF_SPAN = KR_OFF_BAR + KR_TAB + 8;    // ring start of each slot's span (int64, loader only)
constexpr uint32_t KR_OFF_MISC = KR_OFF_SPAN + 8 * KR_NSLOT;   // stage flags, tensor-memory address, abort flag
constexpr size_t KR_SMEM = KR_OFF_MISC + 4 * KR_NB + 16;
constexpr int KR_THREADS = 14 * 32;
static_assert(KR_OFF_RAW % 1024 == 0 && KR_OFF_BAR % 8 == 0 && KR_RING >= KR_BLK * 256 + 8, "shared layout");
static_assert(KR_SMEM <= 232448, "shared memory of the tensor-memory reconstruct kernel");
static_assert(KR_RING * 4 >= 2 * 128 * 128 * 4, "the ring holds the operand table while tensor memory is filled");

// 16 phi_k[p] as split operand words, [precision][pixel half][hi, lo][rank pair q][pixel p % 128]:
// one contiguous 128 KB slice per CTA (64 KB of hi words for plain BF16)
__device__ __align__(16) uint32_t g_kron[3][2][2][128][128];

template <int P>
ABCS_D void kron_setup_p(int q, int p) {
    const int r = p >> 4, c = p & 15;
    double v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int z = zz_pos<16>(2 * q + e);
        v[e] = (double)KR_SCALE * Dd<16>(z >> 4, r) * Dd<16>(z & 15, c);
    }
    uint32_t h, l;
    split2d<P>(v[0], v[1], h, l);
    g_kron[pidx<P>()][p >> 7][0][q][p & 127] = h;
    g_kron[pidx<P>()][p >> 7][1][q][p & 127] = l;
}

__global__ void kron_setup_kernel() {     // grid 128 (rank pairs), block 256 (pixels)
    kron_setup_p<kP16>(blockIdx.x, threadIdx.x);
    kron_setup_p<kPB16>(blockIdx.x, threadIdx.x);
    kron_setup_p<kPB1>(blockIdx.x, threadIdx.x);
}

template <int P>
__global__ void __launch_bounds__(KR_THREADS, 1) recon_umma_kernel(ReconArgs a, int64_t ntot) {
    extern __shared__ __align__(1024) unsigned char kr_smem[];
    unsigned char* smem = kr_smem;
    constexpr bool kSplit = P != kPB1;
    constexpr uint32_t IDESC = umma_idesc_f16(KR_BLK, P != kP16);
    const uint32_t sb = smem_u32(smem), bar = sb + KR_OFF_BAR;
    KrInfo* info = reinterpret_cast<KrInfo*>(smem + KR_OFF_INFO);
    volatile int* sflag = reinterpret_cast<volatile int*>(smem + KR_OFF_MISC);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + KR_OFF_MISC + 4 * KR_NB);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + KR_OFF_MISC + 4 * KR_NB + 4);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int half = blockIdx.x & 1, G2 = gridDim.x >> 1;
    const int64_t T = (ntot + KR_BLK - 1) / KR_BLK, t0 = blockIdx.x >> 1;
    const int my_n = t0 < T ? (int)((T - t0 + G2 - 1) / G2) : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (t == 32) {
        for (int b = 0; b < KR_NSLOT; ++b) {
            mbar_init(bar + KR_RAWF + 8 * b, 1);
            mbar_init(bar + KR_RAWE + 8 * b, 8);
        }
        for (int b = 0; b < KR_NB; ++b) {
            mbar_init(bar + KR_BF + 8 * b, 8);
            mbar_init(bar + KR_BE + 8 * b, 1);
        }
        for (int b = 0; b < KR_NACC; ++b) {
            mbar_init(bar + KR_ACCF + 8 * b, 1);
            mbar_init(bar + KR_ACCE + 8 * b, 4);
        }
        mbar_init(bar + KR_DRAIN, 1);
        mbar_init(bar + KR_TAB, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort_flag = 0;
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    const uint32_t tmem = *tmem_slot;
    // A = 16 Phi_h into tensor memory (hi words in columns 0..127, lo words
    // in 128..255): the CTA's table slice is staged in the (still unused)
    // coefficient ring by one bulk copy
    constexpr uint32_t kTabBytes = (kSplit ? 2 : 1) * 128 * 128 * 4;
    if (t == 32) {
        mbar_arrive_tx(bar + KR_TAB, kTabBytes);
        bulk_g2s(sb + KR_OFF_RAW, &g_kron[pidx<P>()][half][0][0][0], kTabBytes, bar + KR_TAB);
    }
    if (warp >= 10) {
        const int sp = warp & 3;
        int ok = 1;
        if (lane == 0) ok = mbar_wait(bar + KR_TAB, 0, abort_flag, a.status);
        if (__shfl_sync(0xffffffffu, ok, 0)) {
            const uint32_t* tab = reinterpret_cast<const uint32_t*>(smem + KR_OFF_RAW) + 32 * sp + lane;
#pragma unroll 1
            for (int part = 0; part < (kSplit ? 2 : 1); ++part)
#pragma unroll 1
                for (int cb = 0; cb < 4; ++cb) {
                    uint32_t v[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = tab[(part * 128 + cb * 32 + i) * 128];
                    tmem_st32(tmem + ((uint32_t)(32 * sp) << 16) + part * 128 + cb * 32, v);
                }
            tmem_wait_st();
        }
    }
    tc5_fence_before();
    __syncthreads();
    tc5_fence_after();
    griddep_wait();

    if (warp == 1) {
        // ---- loader: tile j's packed coefficients [s0, e) as the 16-byte span
        // [lo4, hi4) placed contiguously in the ring; the converters release
        // tiles in order, and a tile waits for its slot and its ring space
        const bool al16 = (reinterpret_cast<uintptr_t>(a.coeffs) & 15) == 0;
        volatile int64_t* span = reinterpret_cast<volatile int64_t*>(smem + KR_OFF_SPAN);
        float* ring = reinterpret_cast<float*>(smem + KR_OFF_RAW);
        const int64_t total = __ldg(a.offsets + ntot);       // end of the packed vector
        int64_t rpos = 0;                                       // ring position (monotonic, floats) of the next span
        int oldest = 0;                                      // oldest tile not yet released
        constexpr int BPL = KR_BLK / 32;                     // blocks per lane
        int64_t noff[BPL];
        int nm[BPL];
        auto fetch = [&](int jt) {                           // offsets and counts, one tile ahead
            const int64_t fb = (t0 + (int64_t)jt * G2) * KR_BLK;
            const int fn = (int)(ntot - fb < KR_BLK ? ntot - fb : KR_BLK);
#pragma unroll
            for (int h2 = 0; h2 < BPL; ++h2) {
                const int i = lane + 32 * h2;
                noff[h2] = i < fn ? __ldg(a.offsets + fb + i) : 0;
                nm[h2] = i < fn ? __ldg(a.counts + fb + i) : 0;
            }
        };
        if (my_n > 0) fetch(0);
        int j = 0;
        for (; j < my_n; ++j) {
            const int slot = j & (KR_NSLOT - 1);
            const int64_t b0 = (t0 + (int64_t)j * G2) * KR_BLK;
            const int n = (int)(ntot - b0 < KR_BLK ? ntot - b0 : KR_BLK);
            int64_t off[BPL];
            int m[BPL], rel[BPL];
#pragma unroll
            for (int h2 = 0; h2 < BPL; ++h2) {
                off[h2] = noff[h2];
                m[h2] = nm[h2];
            }
            if (j + 1 < my_n) fetch(j + 1);
            const int64_t start = __shfl_sync(0xffffffffu, off[0], 0);
            bool bad = false;
            int end_rel = 0, kmax = 0;
#pragma unroll
            for (int h2 = 0; h2 < BPL; ++h2) {
                rel[h2] = 0;
                if (lane + 32 * h2 >= n) {
                    m[h2] = 0;
                    continue;
                }
                const int64_t r = off[h2] - start;
                if (start < 0 || m[h2] < 0 || m[h2] > 256 || r < 0 || r + m[h2] > KR_BLK * 256 ||
                    start + r + m[h2] > total) {
                    bad = true;
                    m[h2] = 0;
                } else {
                    rel[h2] = (int)r;
                }
                end_rel = max(end_rel, rel[h2] + m[h2]);
                kmax = max(kmax, m[h2]);
            }
            if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(a.status, ABCS_DEV_BADCOUNT);
            end_rel = warp_max(end_rel);
            kmax = warp_max(kmax);
            const int64_t s0 = start < 0 ? 0 : start;
            const int sh = (int)(s0 & 3);
            const int64_t lo4 = s0 - sh, e = s0 + end_rel, hi4 = (e + 3) & ~(int64_t)3, sz = hi4 - lo4;
            if ((rpos % KR_RING) + sz > KR_RING) rpos += KR_RING - (rpos % KR_RING);
            bool ok = true;
            while (oldest < j && (j - oldest >= KR_NSLOT || rpos + sz - span[oldest & (KR_NSLOT - 1)] > KR_RING)) {
                int w = 1;
                if (lane == 0)
                    w = mbar_wait(bar + KR_RAWE + 8 * (oldest & (KR_NSLOT - 1)), (oldest / KR_NSLOT) & 1, abort_flag,
                                  a.status);
                if (!__shfl_sync(0xffffffffu, w, 0)) {
                    ok = false;
                    break;
                }
                ++oldest;
            }
            if (!ok) break;
            const int ro = (int)(rpos % KR_RING);
            KrInfo& I = info[slot];
#pragma unroll
            for (int h2 = 0; h2 < BPL; ++h2) {
                I.rel[lane + 32 * h2] = ro + sh + rel[h2];
                I.m[lane + 32 * h2] = m[h2];
            }
            if (lane == 0) {
                I.nst = kmax > 0 ? (kmax + KR_KS - 1) / KR_KS : 1;
                span[slot] = rpos;
            }
            // bulk part [lo4, x1); plain loads for the last ragged 16 bytes of
            // the packed vector (a rounded span would read past it) or for an
            // unaligned coefficient pointer
            int64_t x1 = hi4 > total ? (e & ~(int64_t)3) : hi4;
            if (!al16) x1 = lo4;
            for (int64_t x = (x1 > s0 ? x1 : s0) + lane; x < e; x += 32) ring[ro + (x - lo4)] = __ldg(a.coeffs + x);
            __syncwarp();
            if (lane == 0) {
                const uint32_t full = bar + KR_RAWF + 8 * slot;
                if (x1 > lo4) {
                    const uint32_t bytes = (uint32_t)(x1 - lo4) * 4u;
                    mbar_arrive_tx(full, bytes);
                    bulk_g2s(sb + KR_OFF_RAW + (uint32_t)ro * 4u, a.coeffs + lo4, bytes, full);
                } else {
                    mbar_arrive(full);
                }
            }
            rpos += sz;
        }
        // copies still in flight land before the CTA leaves
        if (lane == 0)
            for (int jj = j > KR_NSLOT ? j - KR_NSLOT : 0; jj < j; ++jj)
                mbar_drain(bar + KR_RAWF + 8 * (jj & (KR_NSLOT - 1)), (jj / KR_NSLOT) & 1, a.status);
    } else if (warp >= 2 && warp < 10) {
        // ---- converters
        const int i = (t - 64) % KR_BLK, part = (t - 64) / KR_BLK;
        int g = 0;
        for (int j = 0; j < my_n; ++j) {
            const int slot = j & (KR_NSLOT - 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar + KR_RAWF + 8 * slot, (j / KR_NSLOT) & 1, abort_flag, a.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const KrInfo& I = info[slot];
            const int nst = I.nst, m = I.m[i];
            const float* raw = reinterpret_cast<const float*>(smem + KR_OFF_RAW) + I.rel[i];
            bool alive = true;
            for (int s = 0; s < nst; ++s, ++g) {
                const int b = g & (KR_NB - 1);
                if (lane == 0) ok = mbar_wait(bar + KR_BE + 8 * b, ((g / KR_NB) & 1) ^ 1, abort_flag, a.status);
                if (!__shfl_sync(0xffffffffu, ok, 0)) {
                    alive = false;
                    break;
                }
#pragma unroll
                for (int cc = 0; cc < KR_CPT; ++cc) {
                    const int c = part * KR_CPT + cc, k0 = KR_KS * s + 8 * c;
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = k0 + e < m ? raw[k0 + e] : 0.f;
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if constexpr (kSplit) split2<P>(v[2 * q], v[2 * q + 1], hi[q], lo[q]);
                        else hi[q] = pk<P>(v[2 * q], v[2 * q + 1]);
                    }
                    unsigned char* st = smem + KR_OFF_STAGE + b * KR_STAGE + c * KR_CHUNK + i * 16;
                    *reinterpret_cast<uint4*>(st) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    if constexpr (kSplit)
                        *reinterpret_cast<uint4*>(st + KR_CH * KR_CHUNK) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    if (warp == 2) sflag[b] = (s == 0 ? 1 : 0) | (s == nst - 1 ? 2 : 0);
                    mbar_arrive(bar + KR_BF + 8 * b);
                }
            }
            if (!alive) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar + KR_RAWE + 8 * slot);
        }
    } else if (warp == 0) {
        // ---- MMA issuer
        if (lane == 0) {
            int g = 0;
            bool alive = true;
            for (int j = 0; j < my_n && alive; ++j) {
                const int acc = j & (KR_NACC - 1);
                if (!mbar_wait(bar + KR_ACCE + 8 * acc, ((j / KR_NACC) & 1) ^ 1, abort_flag, a.status)) break;
                tc5_fence_after();
                const uint32_t d = tmem + 256 + KR_BLK * acc;
                for (int s = 0;; ++s) {
                    const int b = g & (KR_NB - 1);
                    if (!mbar_wait(bar + KR_BF + 8 * b, (g / KR_NB) & 1, abort_flag, a.status)) {
                        alive = false;
                        break;
                    }
                    tc5_fence_after();
                    const int f = sflag[b];
                    const uint32_t st = sb + KR_OFF_STAGE + b * KR_STAGE;
#pragma unroll
                    for (int kk = 0; kk < KR_KS / 16; ++kk) {
                        const uint32_t ah = tmem + 8 * ((KR_KS / 16 * s + kk) & 15);
                        const uint64_t bh = umma_desc(st + 2 * kk * KR_CHUNK, KR_CHUNK, 128);
                        umma_tmem_a(d, ah, bh, IDESC, (f & 1) && kk == 0 ? 0u : 1u);
                        if constexpr (kSplit) {
                            const uint64_t bl = umma_desc(st + KR_CH * KR_CHUNK + 2 * kk * KR_CHUNK, KR_CHUNK, 128);
                            umma_tmem_a(d, ah + 128, bh, IDESC, 1u);
                            umma_tmem_a(d, ah, bl, IDESC, 1u);
                        }
                    }
                    umma_commit(bar + KR_BE + 8 * b);     // the stage buffer is free once these complete
                    ++g;
                    if ((f & 2) || s == 256 / KR_KS - 1) {
                        umma_commit(bar + KR_ACCF + 8 * acc);   // the tile's accumulator is ready
                        break;
                    }
                }
            }
            umma_commit(bar + KR_DRAIN);
            mbar_drain(bar + KR_DRAIN, 0, a.status);
        }
        __syncwarp();
    } else {
        // ---- epilogue
        const int sp = warp & 3, p = 128 * half + 32 * sp + lane;
        const ImgGeom& G = a.g;
        const int64_t pix = (int64_t)(p >> 4) * G.Wc + (p & 15);
        auto u8 = [](float v) { return (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f); };
        for (int j = 0; j < my_n; ++j) {
            const int acc = j & (KR_NACC - 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar + KR_ACCF + 8 * acc, (j / KR_NACC) & 1, abort_flag, a.status);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc5_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * sp) << 16) + 256 + KR_BLK * acc;
            const int64_t b0 = (t0 + (int64_t)j * G2) * KR_BLK;
            const int n = (int)(ntot - b0 < KR_BLK ? ntot - b0 : KR_BLK);
            int k, bi, bj;
            block_coords(G, b0, k, bi, bj);
            int64_t pos = (int64_t)k * G.Hc * G.Wc + (int64_t)(bi * 16) * G.Wc + bj * 16 + pix;
#pragma unroll 1
            for (int g32 = 0; g32 < KR_BLK / 32; ++g32) {
                uint32_t v[32];
                tmem_ld32(ta + 32 * g32, v);
                if (g32 == KR_BLK / 32 - 1) {       // the accumulator is free for the next tile
                    tc5_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar + KR_ACCE + 8 * acc);
                }
#pragma unroll
                for (int ii = 0; ii < 32; ++ii) {
                    if (32 * g32 + ii < n) {
                        const float x = __uint_as_float(v[ii]) * (1.f / KR_SCALE);
                        if (a.out) a.out[pos] = x;
                        if (a.out_u8) a.out_u8[pos] = u8(x);
                    }
                    pos += 16;
                    if (++bj == G.nbw) {          // next block row (or the next image's first)
                        bj = 0;
                        pos += 15 * (int64_t)G.Wc;
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

// ---------------------------------------------------------------------------
// sense: C = D X D^T, computed transposed.  Stage 1 V = D X^T (A = D with
// its columns permuted, B = X^T read from the staged pixels) is the row
// transform of every pixel row; stage 2 R = V D^T (A = V from the
// accumulators, B = D^T constant) gives R[v][u] = C[u][v].
// K-permutation of stage 1: MMA k = 2q + e, 2q + 8 + e (e = 0, 1) stands for
// pixel column 4q + e, 4q + 2 + e, so each lane's B fragment of one pixel
// row is 4 consecutive bytes (one 32-bit shared load).  Pixels sit in shared
// memory block after block, 16 bytes per row, which makes those loads
// bank-conflict free.  The block's first
// m_i zigzag coefficients are scattered into the segment's packed staging
// buffer and the whole segment range is written out with 16-byte stores.
// ---------------------------------------------------------------------------

// two pixels (bytes `hi2` * 2 and * 2 + 1 of w) as an operand pair; exact
template <int P>
ABCS_D uint32_t px_pair(uint32_t w, int hi2) {
    if constexpr (P == kP16) {
        // 0x64XX as FP16 is 1024 + XX exactly; subtract 1024
        const uint32_t v = __byte_perm(w, 0x64646464u, hi2 ? 0x4342 : 0x4140);
        __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&v), __halves2half2(__ushort_as_half(0x6400),
                                                                                 __ushort_as_half(0x6400)));
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        const int b0 = (w >> (16 * hi2)) & 0xFF, b1 = (w >> (16 * hi2 + 8)) & 0xFF;
        return pk<P>((float)b0, (float)b1);
    }
}

// Image bases of the CTA's images k_first .. k_first + SK_MAX - 1 (when the
// allocation does not write them): warp 0 sums the totals of the images
// before k_first and scans those of the CTA's images into kbase[].
constexpr int SK_MAX = 64;
ABCS_D void cta_image_bases(const SenseArgs& a, int k_first, int64_t* kbase) {
    const int lane = threadIdx.x & 31;
    int64_t v = 0;
    for (int k = lane; k < k_first; k += 32) v += __ldg(a.img_total + k);
    int64_t carry = warp_sum(v);
#pragma unroll
    for (int h = 0; h < SK_MAX / 32; ++h) {
        const int k = k_first + 32 * h + lane;
        const int64_t t = k < a.g.n_img ? __ldg(a.img_total + k) : 0;
        int64_t incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        kbase[32 * h + lane] = carry + incl - t;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// counts and image-local offsets from the allocation, image bases from its
// last CTA or from the CTA's own table; pos = byte offset of the block's
// top-left pixel in the input
ABCS_D MetaRaw sense_meta_load(const SenseArgs& a, const SegGeom& sg, const int64_t* kbase, int k_first) {
    const int lane = threadIdx.x & 31;
    MetaRaw r;
    r.off = 0;
    r.pos = 0;
    r.m = 0;
    if (lane < sg.nblk) {
        const int64_t b = sg.b0 + lane;
        int k, bi, bj;
        block_coords(a.g, b, k, bi, bj);
        r.off = __ldg(a.offsets + b) + (a.pilot_bases ? __ldg(a.img_base + k) : kbase[k - k_first]);
        r.m = __ldg(a.counts + b);
        r.pos = (int64_t)k * a.g.img_stride + (int64_t)(bi * 16) * a.g.pitch + bj * 16;
    }
    return r;
}

// pixel positions only (they do not depend on the allocation)
ABCS_D void sense_pos_store(const SenseArgs& a, const SegGeom& sg, SegMeta<SEG>& M) {
    const int lane = threadIdx.x & 31;
    if (lane < sg.nblk) {
        int k, bi, bj;
        block_coords(a.g, sg.b0 + lane, k, bi, bj);
        M.pos[lane] = (int64_t)k * a.g.img_stride + (int64_t)(bi * 16) * a.g.pitch + bj * 16;
    }
    if (lane == 0) M.sg = sg;
}

ABCS_D void sense_meta_store(const SegGeom& sg, const MetaRaw& r, SegMeta<SEG>& M) {
    const int lane = threadIdx.x & 31;
    const int64_t start = __shfl_sync(0xffffffffu, r.off, 0);
    const int rel = (int)(r.off - start);
    const int end = warp_max(lane < sg.nblk ? rel + r.m : 0);
    M.rel[lane] = rel;
    M.cnt[lane] = r.m;
    M.pos[lane] = r.pos;
    if (lane == 0) {
        M.start = start;
        M.n = end;
        M.sh = (int)(start & 3);
        M.sg = sg;
    }
}

// all threads: copy the pixels of the segment's blocks, block c's row r
// (16 bytes) to 256 c + 16 r
ABCS_D void sense_pixels(const SenseArgs& a, const SegMeta<SEG>& M, uint8_t* dst, bool vec) {
#pragma unroll
    for (int h = 0; h < SEG * 16 / 256; ++h) {
        const int id = threadIdx.x + 256 * h, c = id >> 4, r = id & 15;
        if (c >= M.sg.nblk) continue;
        const uint8_t* src = a.img + M.pos[c] + (int64_t)r * a.g.pitch;
        uint8_t* d = dst + 256 * c + 16 * r;
        if (vec) {
            const unsigned sd = (unsigned)__cvta_generic_to_shared(d);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sd), "l"(src) : "memory");
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) d[i] = __ldg(src + i);
        }
    }
}

template <int P>
__global__ void __launch_bounds__(256, 4) sense_tc_kernel(SenseArgs a, int64_t ntot) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint8_t (*pix)[16 * SEG * 16] = reinterpret_cast<uint8_t (*)[16 * SEG * 16]>(smem);
    float* ost = reinterpret_cast<float*>(smem + SNB * 16 * SEG * 16);
    SegMeta<SEG>* meta = reinterpret_cast<SegMeta<SEG>*>(smem + SNB * 16 * SEG * 16 + kSegFloats * sizeof(float));
    const int warp = threadIdx.x >> 5;
    const Frag f;
    uint32_t DAh[4], DAl[4], DTh[2][2], DTl[2][2];
    frag_a<P>(kSetSenseA, DAh, DAl);
    frag_b<P>(kSetSenseB, DTh, DTl);
    // 4 x the ranks of R[g + 8 (i>>1)][2q + (i&1) + 8 nt] = C[u = 2q + (i&1) + 8 nt][v = g + 8 (i>>1)]
    // (byte offsets in the segment's packed staging buffer)
    int rkb[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rkb[nt][i] = 4 * zz_rank(2 * f.q + (i & 1) + 8 * nt, f.g + 8 * (i >> 1), 16);

    const ImgGeom& g = a.g;
    const bool vec = ((reinterpret_cast<uintptr_t>(a.img) | (uintptr_t)g.pitch |
                       (uintptr_t)(g.n_img > 1 ? g.img_stride : 0)) & 15) == 0;
    int64_t r0, r1;
    cta_range(ntot, &r0, &r1);
    const int nseg = (int)((r1 - r0 + SEG - 1) / SEG);
    if (nseg <= 0) return;
    // the first segment's pixels do not depend on the allocation: they are
    // staged before the wait for the pilot kernel, which lets this grid start
    // once it has passed its own wait (so the images are final by then)
    if (warp == 0) sense_pos_store(a, seg_geom<SEG>(r0, r1, 0), meta[0]);
    __syncthreads();
    sense_pixels(a, meta[0], pix[0], vec);
    cp_async_commit();
    griddep_wait();
    __shared__ int64_t kbase[SK_MAX];
    const int k_first = (int)(r0 / g.n_blocks);
    if (!a.pilot_bases && warp == 0) cta_image_bases(a, k_first, kbase);
    __syncthreads();                            // meta[0] is rewritten below
    // pixels of segments j + 1 .. j + SDEPTH are in flight while segment j is
    // transformed (the same rings as in reconstruct)
    MetaRaw raw;
    if (warp == 0) {
        for (int d = 0; d < SDEPTH && d < nseg; ++d)
            sense_meta_store(seg_geom<SEG>(r0, r1, d), sense_meta_load(a, seg_geom<SEG>(r0, r1, d), kbase, k_first),
                             meta[d]);
        if (SDEPTH < nseg) raw = sense_meta_load(a, seg_geom<SEG>(r0, r1, SDEPTH), kbase, k_first);
    }
    __syncthreads();
#pragma unroll
    for (int d = 1; d < SDEPTH; ++d) {
        if (d < nseg) sense_pixels(a, meta[d], pix[d], vec);
        cp_async_commit();
    }
    int mi = 0, bi = 0, mn = SDEPTH % SNM, bn = SDEPTH % SNB;
    for (int j = 0; j < nseg; ++j) {
        const int jn = j + SDEPTH;
        if (jn < nseg && warp == 0) {
            sense_meta_store(seg_geom<SEG>(r0, r1, jn), raw, meta[mn]);
            if (jn + 1 < nseg) raw = sense_meta_load(a, seg_geom<SEG>(r0, r1, jn + 1), kbase, k_first);
        }
        cp_async_wait_group<SDEPTH - 1>();
        __syncthreads();
        if (jn < nseg) sense_pixels(a, meta[mn], pix[bn], vec);
        cp_async_commit();

        const SegMeta<SEG>& M = meta[mi];
        const int nblk = M.sg.nblk;
        const uint8_t* px = pix[bi];
        const uint32_t os = smem_u32(ost + M.sh);
#pragma unroll 2
        for (int c = warp; c < nblk; c += 8) {
            uint32_t xb[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int y = f.g + 8 * nt;    // bank 4 g + q: conflict free
                const uint32_t w = *reinterpret_cast<const uint32_t*>(px + 256 * c + 16 * y + 4 * f.q);
                xb[nt][0] = px_pair<P>(w, 0);
                xb[nt][1] = px_pair<P>(w, 1);
            }
            float V[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma0<P>(V[nt], DAh, xb[nt][0], xb[nt][1]);
                if constexpr (P != kPB1) mma<P>(V[nt], DAl, xb[nt][0], xb[nt][1]);
            }
            uint32_t Ah[4], Al[4];
            split2<P>(V[0][0], V[0][1], Ah[0], Al[0]);
            split2<P>(V[0][2], V[0][3], Ah[1], Al[1]);
            split2<P>(V[1][0], V[1][1], Ah[2], Al[2]);
            split2<P>(V[1][2], V[1][3], Ah[3], Al[3]);
            float R[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
                mma_split<P>(R[nt], Ah, Al, DTh[nt][0], DTh[nt][1], DTl[nt][0], DTl[nt][1]);
            const int m4 = 4 * M.cnt[c];
            const uint32_t ob = os + 4u * (uint32_t)M.rel[c];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i) sts_f_lt(ob + (uint32_t)rkb[nt][i], R[nt][i], rkb[nt][i], m4);
        }
        __syncthreads();
        // copy-out of the segment's packed range and its global offsets
        const int64_t start = M.start;
        int n = M.n;
        if (start + n > a.capacity) {
            if (threadIdx.x == 0) set_status(a.status, ABCS_DEV_CAPACITY);
            n = start < a.capacity ? (int)(a.capacity - start) : 0;
        }
        stage_out(ost, a.coeffs, start, n);
        if (threadIdx.x < nblk) {
            const int64_t b = M.sg.b0 + threadIdx.x;
            a.offsets[b] = start + M.rel[threadIdx.x];
            if (b == ntot - 1) a.offsets[ntot] = start + M.n;
        }
        mi = mi + 1 == SNM ? 0 : mi + 1;
        bi = bi + 1 == SNB ? 0 : bi + 1;
        mn = mn + 1 == SNM ? 0 : mn + 1;
        bn = bn + 1 == SNB ? 0 : bn + 1;
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// DD pilot on the tensor cores (Alg. 2, B = 16): n_i = #{rank j < m1 :
// |c_j| > T}, decided on the exact coefficient.  One CTA per 32-block tile
// of a block row (warp w takes blocks w, w + 8, w + 16, w + 24, all their
// pixels loaded up front), one partial sum per tile, the fused allocation
// of dd_pilot_kernel; each block's coefficients come from the sensing transform's
// FP16x2 fragments (pixels exact in FP16, D split hi + lo).  A coefficient
// within the band E_tc of T is recomputed in FP32 by the whole warp from the
// block's pixels, which its lanes already hold (8 each): lane terms
// fl(D_u,n D_v,m) x_n,m, summed in an FMA chain of 8 and a 5-level shuffle
// tree; with the FP32 table's rounding that is within 16 2^-24 S of c, and
// the band E_32 = 32 2^-24 S decides.  Inside E_32 the warp decides exactly
// (dd_exact_warp16): integers at (u, v) in {0, 8}^2, else FP64 within
// 1e-11, with the same 1e-9 ambiguity rule as the FP32 pilot.
// Band: with S = 255 B bounding sum |D_u,n| |X_n,m| |D_v,m| (each row of D has
// unit L2 norm, so its L1 norm is at most sqrt(B)), the hi + lo split of D
// and of the stage-1 result (each within 2^-22 relative, or 2^-25 absolute in
// FP16's subnormal range), the missing lo x lo product (2^-22) and FP32
// accumulation of 32 + 48 terms (each addition within 2^-23 relative, which
// also covers truncating adders) give |c_tc - c| <= 88 2^-23 S + 2^-25 16 S
// / 255; E_tc doubles the first term and takes 0.01 for the second.
// ---------------------------------------------------------------------------
// Exact |c(u,v)| > T of the block whose pixels the warp holds (lane (g, q):
// pw[h] = row g + 8 h, columns 4q .. 4q + 3); every lane returns the decision.
ABCS_D bool dd_exact_warp16(int u, int v, const uint32_t (&pw)[2], int T, uint32_t* status) {
    const Frag f;
    if ((u == 0 || u == 8) && (v == 0 || v == 8)) {       // c = S / 16 with integer S
        int S = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int su = rational_sign<16>(u, f.g + 8 * h);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                S += su * rational_sign<16>(v, 4 * f.q + cc) * (int)((pw[h] >> (8 * cc)) & 0xFFu);
        }
        S = warp_sum(S);
        return abs(S) > T * 16;
    }
    double c = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const double du = Dd<16>(u, f.g + 8 * h);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
            c = fma(du * Dd<16>(v, 4 * f.q + cc), (double)((pw[h] >> (8 * cc)) & 0xFFu), c);
    }
    c = __shfl_sync(0xffffffffu, warp_sum(c), 0);
    const double d = fabs(c) - (double)T;
    if (fabs(d) <= 1e-9) {
        if ((threadIdx.x & 31) == 0) set_status(status, ABCS_DEV_AMBIGUOUS);
        return false;
    }
    return d > 0.0;
}

constexpr int kDdNB = 32, kDdBPW = kDdNB / 8;   // blocks of a CTA's tile (one block row), per warp

__global__ void __launch_bounds__(256, 3) dd_pilot_tc_kernel(SenseArgs a) {
    __shared__ unsigned long long sh[32];
    __shared__ int64_t sh2[33];
    __shared__ int64_t sW;
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Frag f;
    uint32_t DAh[4], DAl[4], DTh[2][2], DTl[2][2];
    frag_a<kP16>(kSetSenseA, DAh, DAl);
    frag_b<kP16>(kSetSenseB, DTh, DTl);
    int rk[2][4];   // ranks of R[g + 8 (i>>1)][2q + (i&1) + 8 nt] = C[u = 2q + (i&1) + 8 nt][v = g + 8 (i>>1)]
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rk[nt][i] = zz_rank(2 * f.q + (i & 1) + 8 * nt, f.g + 8 * (i >> 1), 16);
    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * kDdNB;
    const int nblk = min(kDdNB, g.nbw - bj0);
    const uint8_t* img = a.img + (int64_t)k * g.img_stride + (int64_t)(bi * 16) * g.pitch;
    constexpr float kS = 255.f * 16.f;
    const float band = 176.f * 1.1920929e-7f * kS + 0.01f;
    const float band32 = 32.f * 5.9604645e-8f * kS;
    const float T = (float)a.T;
    const int m1 = a.m1;
    griddep_wait();
    // every block's pixels first (pwj[j][h]: block warp + 8 j, row g + 8 h, columns 4q .. 4q + 3)
    uint32_t pwj[kDdBPW][2];
#pragma unroll
    for (int j = 0; j < kDdBPW; ++j)
#pragma unroll
        for (int h = 0; h < 2; ++h)
            pwj[j][h] = warp + 8 * j < nblk
                            ? __ldg(reinterpret_cast<const uint32_t*>(img + (bj0 + warp + 8 * j) * 16 +
                                                                      (int64_t)(f.g + 8 * h) * g.pitch + 4 * f.q))
                            : 0u;
    unsigned long long mine = 0;
#pragma unroll 1
    for (int j = 0; j < kDdBPW; ++j) {
        const int c = warp + 8 * j;
        if (c >= nblk) break;
        uint32_t xb[2][2], pw[2];       // pw[h]: pixels of row g + 8 h, columns 4q .. 4q + 3
        // the next block's pixels move to the front (fixed register names)
        pw[0] = pwj[0][0];
        pw[1] = pwj[0][1];
#pragma unroll
        for (int jj = 0; jj + 1 < kDdBPW; ++jj) {
            pwj[jj][0] = pwj[jj + 1][0];
            pwj[jj][1] = pwj[jj + 1][1];
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            xb[nt][0] = px_pair<kP16>(pw[nt], 0);
            xb[nt][1] = px_pair<kP16>(pw[nt], 1);
        }
        float V[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            mma0<kP16>(V[nt], DAh, xb[nt][0], xb[nt][1]);
            mma<kP16>(V[nt], DAl, xb[nt][0], xb[nt][1]);
        }
        uint32_t Ah[4], Al[4];
        split2<kP16>(V[0][0], V[0][1], Ah[0], Al[0]);
        split2<kP16>(V[0][2], V[0][3], Ah[1], Al[1]);
        split2<kP16>(V[1][0], V[1][1], Ah[2], Al[2]);
        split2<kP16>(V[1][2], V[1][3], Ah[3], Al[3]);
        float R[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
            mma_split<kP16>(R[nt], Ah, Al, DTh[nt][0], DTh[nt][1], DTl[nt][0], DTl[nt][1]);
        int n = 0;
        uint32_t pend = 0;              // bit 4 nt + i: coefficient inside the band
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (rk[nt][i] >= m1) continue;
                const float v = fabsf(R[nt][i]);
                if (v > T + band) ++n;
                else if (v >= T - band) pend |= 1u << (4 * nt + i);
            }
        // in-band coefficients, one at a time over the warp
        for (unsigned any = __ballot_sync(0xffffffffu, pend != 0); any;
             any = __ballot_sync(0xffffffffu, pend != 0)) {
            const int src = __ffs(any) - 1;
            const uint32_t pb = __shfl_sync(0xffffffffu, pend, src);
            const int e = __ffs(pb) - 1, nt = e >> 2, i = e & 3;
            const int u = 2 * (src & 3) + (i & 1) + 8 * nt, vv = (src >> 2) + 8 * (i >> 1);
            float p = 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float du = Dc<16>(u, f.g + 8 * h);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    p = fmaf(du * Dc<16>(vv, 4 * f.q + cc), (float)((pw[h] >> (8 * cc)) & 0xFFu), p);
            }
            const float v = fabsf(__shfl_sync(0xffffffffu, warp_sum(p), src));   // the same in every lane
            bool hit = v > T + band32;
            if (!hit && v >= T - band32) hit = dd_exact_warp16(u, vv, pw, a.T, a.status);
            if (lane == src) {
                n += hit ? 1 : 0;
                pend &= ~(1u << e);
            }
        }
        n = __reduce_add_sync(0xffffffffu, n);
        if (lane == 0) {
            a.w[(int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0 + c] = n;
            mine += (unsigned long long)n;
        }
    }
    mine = block_sum(mine, sh);
    if (threadIdx.x == 0)
        a.wpart[(int64_t)k * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = mine;
    pilot_alloc_tail(a, 2, k, gridDim.x * gridDim.y, sh2, &sW, &s_last);
}

// one CTA per segment at most, and no more CTAs than fit on the GPU at once
template <typename K>
cudaError_t grid_segs(K kernel, int64_t ntot, int seg, size_t smem, int* grid) {
    const int64_t nseg = (ntot + seg - 1) / seg;
    int dev, sms, per_sm;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
    if (e) return e;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (int)(nseg < cap ? nseg : cap);
    return cudaSuccess;
}

template <int P>
cudaError_t launch_recon_umma_p(const ReconArgs& a, cudaStream_t s) {
    const int64_t ntot = (int64_t)a.g.n_img * a.g.n_blocks;
    if (ntot <= 0) return cudaSuccess;
    int dev, sms;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaFuncSetAttribute(recon_umma_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KR_SMEM);
    if (e) return e;
    const int64_t T = (ntot + KR_BLK - 1) / KR_BLK;
    const int pairs = (int)(T < sms / 2 ? T : (sms / 2 > 0 ? sms / 2 : 1));
    return launch_pdl(recon_umma_kernel<P>, dim3(2 * pairs), dim3(KR_THREADS), KR_SMEM, s, a, ntot);
}

// ABCS_RECON_TC=umma selects the tensor-memory kernel (measured slower than
// the mma.sync one on the 64 x 512^2 workload, so not the default)
inline bool recon_umma_selected() {
    const char* v = getenv("ABCS_RECON_TC");
    return v && strcmp(v, "umma") == 0;
}

template <int P>
cudaError_t launch_recon_tc_p(const ReconArgs& a, cudaStream_t s) {
    if (recon_umma_selected()) return launch_recon_umma_p<P>(a, s);
    const int64_t ntot = (int64_t)a.g.n_img * a.g.n_blocks;
    int grid = 0;
    cudaError_t e = grid_segs(recon_tc_kernel<P>, ntot, RSEG, kReconSmem, &grid);
    if (e) return e;
    return launch_pdl(recon_tc_kernel<P>, dim3(grid), dim3(256), kReconSmem, s, a, ntot);
}

template <int P>
cudaError_t launch_sense_tc_p(const SenseArgs& a, cudaStream_t s) {
    const int64_t ntot = (int64_t)a.g.n_img * a.g.n_blocks;
    int grid = 0;
    cudaError_t e = grid_segs(sense_tc_kernel<P>, ntot, SEG, kSenseSmem, &grid);
    if (e) return e;
    return launch_pdl(sense_tc_kernel<P>, dim3(grid), dim3(256), kSenseSmem, s, a, ntot);
}

// The image bases of a CTA's range fit its table when no range of
// ceil(ntot / grid) blocks spans more than SK_MAX images.
bool sense_tc_bases_fit(const SenseArgs& a) {
    const int64_t ntot = (int64_t)a.g.n_img * a.g.n_blocks;
    int grid = 0;
    if (grid_segs(sense_tc_kernel<kP16>, ntot, SEG, kSenseSmem, &grid) != cudaSuccess || grid <= 0) return false;
    const int64_t per = (ntot + grid - 1) / grid;
    return (per + a.g.n_blocks - 1) / a.g.n_blocks + 1 <= SK_MAX;
}
}  // namespace

cudaError_t setup_tc_fragments() {
    tc_frag_setup_kernel<<<1, 32>>>();
    kron_setup_kernel<<<128, 256>>>();
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaDeviceSynchronize();
    return e;
}

cudaError_t launch_recon_tc(const ReconArgs& a, cudaStream_t s) {
    if (a.g.B != 16) return cudaErrorInvalidValue;
    switch (a.precision) {
        case kP16: return launch_recon_tc_p<kP16>(a, s);
        case kPB16: return launch_recon_tc_p<kPB16>(a, s);
        case kPB1: return launch_recon_tc_p<kPB1>(a, s);
    }
    return cudaErrorInvalidValue;
}

// the tensor-core DD pilot reads each block row's 16 pixels as 4-byte words
bool dd_tc_usable(const SenseArgs& a) {
    const uintptr_t al = reinterpret_cast<uintptr_t>(a.img) | (uintptr_t)a.g.pitch |
                         (uintptr_t)(a.g.n_img > 1 ? a.g.img_stride : 0);
    return a.g.B == 16 && (al & 3) == 0;
}

cudaError_t launch_dd_tc_alloc(const SenseArgs& a, cudaStream_t s) {
    if (!dd_tc_usable(a)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((a.g.nbw + kDdNB - 1) / kDdNB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(dd_pilot_tc_kernel, grid, dim3(256), 0, s, a);
}

bool sense_tc_bases_in_kernel(const SenseArgs& a) { return a.g.B == 16 && sense_tc_bases_fit(a); }

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
