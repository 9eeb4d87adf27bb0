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

// d += a * b on the tensor cores (m16n8k16, FP32 accumulate)
template <int P>
ABCS_D void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (P == kP16) {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// d = a * b (zero accumulator)
template <int P>
ABCS_D void mma0(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    const float z = 0.f;
    if constexpr (P == kP16) {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%10,%10,%10,%10};\n"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(z));
    } else {
        asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%10,%10,%10,%10};\n"
            : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(z));
    }
}

// d = A * B with both operands split (3 products) or single (1 product)
template <int P>
ABCS_D void mma_split(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                      uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma0<P>(d, ah, bh0, bh1);
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

// Operand fragments of the constant factors D and D^T (hi and lo words), per
// precision, fragment set and lane.  They are split from the FP64 table once
// per device by tc_frag_setup_kernel: doing it in every CTA's prologue kept
// the narrow FP64 pipe of this GPU busy for a large part of each launch.
enum { kSetSenseA = 0, kSetSenseB = 1, kSetReconA = 2, kSetReconB = 3 };
__device__ uint32_t g_tc_frag[3][4][8][32];

template <int P>
__host__ __device__ constexpr int pidx() { return P == kP16 ? 0 : (P == kPB16 ? 1 : 2); }

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
constexpr int SEG = 32;                        // sensing segment (blocks)
constexpr int RSEG = 32;                       // reconstruction segment (blocks)
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
constexpr size_t kReconSmem = 2 * kRSegFloats * sizeof(float) + 3 * sizeof(SegMeta<RSEG>);
constexpr size_t kSenseSmem = 2 * 16 * SEG * 16 + kSegFloats * sizeof(float) + 3 * sizeof(SegMeta<SEG>);

template <int P>
__global__ void __launch_bounds__(256, 3) recon_tc_kernel(ReconArgs a, int64_t ntot) {
    extern __shared__ __align__(16) unsigned char smem[];
    float (*stage)[kRSegFloats] = reinterpret_cast<float (*)[kRSegFloats]>(smem);
    SegMeta<RSEG>* meta = reinterpret_cast<SegMeta<RSEG>*>(smem + 2 * kRSegFloats * sizeof(float));
    const int warp = threadIdx.x >> 5;
    const Frag f;
    uint32_t ATh[4], ATl[4], DBh[2][2], DBl[2][2];
    frag_a<P>(kSetReconA, ATh, ATl);
    frag_b<P>(kSetReconB, DBh, DBl);
    // ranks of the 8 coefficients this lane feeds into B = C: (2q + e, g + 8 nt), e in {0,1,8,9}
    int rk[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rk[nt][i] = zz_rank(2 * f.q + (i & 1) + 8 * (i >> 1), f.g + 8 * nt, 16);

    griddep_wait();
    const ImgGeom& g = a.g;
    int64_t r0, r1;
    cta_range(ntot, &r0, &r1);
    const int nseg = (int)((r1 - r0 + RSEG - 1) / RSEG);
    if (nseg <= 0) return;
    const int lo = f.g * g.Wc + 2 * f.q;
    MetaRaw raw;
    if (warp == 0) {
        recon_meta_store(a, seg_geom<RSEG>(r0, r1, 0), recon_meta_load(a, seg_geom<RSEG>(r0, r1, 0)), meta[0]);
        if (1 < nseg) raw = recon_meta_load(a, seg_geom<RSEG>(r0, r1, 1));
    }
    __syncthreads();
    stage_in_async(stage[0], a.coeffs, meta[0].start, meta[0].n);
    cp_async_commit();
    int mi = 0;                                 // meta slot of segment j (j mod 3)
    for (int j = 0; j < nseg; ++j) {
        const int mn = mi == 2 ? 0 : mi + 1;
        if (j + 1 < nseg && warp == 0) {
            recon_meta_store(a, seg_geom<RSEG>(r0, r1, j + 1), raw, meta[mn]);
            if (j + 2 < nseg) raw = recon_meta_load(a, seg_geom<RSEG>(r0, r1, j + 2));
        }
        cp_async_wait_all();
        __syncthreads();
        if (j + 1 < nseg) stage_in_async(stage[(j + 1) & 1], a.coeffs, meta[mn].start, meta[mn].n);
        cp_async_commit();

        const SegMeta<RSEG>& M = meta[mi];
        const SegGeom sg = M.sg;
        const float* st = stage[j & 1] + M.sh;
#pragma unroll
        for (int c = warp; c < sg.nblk; c += 8) {
            const int m = M.cnt[c];
            const float* sb = st + M.rel[c];
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                float cv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) cv[i] = (rk[nt][i] < m) ? sb[rk[nt][i]] : 0.f;
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
        mi = mn;
    }
    cp_async_wait_all();
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

// counts and image-local offsets from the allocation, image bases from its
// last CTA; pos = byte offset of the block's top-left pixel in the input
ABCS_D MetaRaw sense_meta_load(const SenseArgs& a, const SegGeom& sg) {
    const int lane = threadIdx.x & 31;
    MetaRaw r;
    r.off = 0;
    r.pos = 0;
    r.m = 0;
    if (lane < sg.nblk) {
        const int64_t b = sg.b0 + lane;
        int k, bi, bj;
        block_coords(a.g, b, k, bi, bj);
        r.off = __ldg(a.offsets + b) + __ldg(a.img_base + k);
        r.m = __ldg(a.counts + b);
        r.pos = (int64_t)k * a.g.img_stride + (int64_t)(bi * 16) * a.g.pitch + bj * 16;
    }
    return r;
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
    float* ost = reinterpret_cast<float*>(smem + 2 * 16 * SEG * 16);
    SegMeta<SEG>* meta = reinterpret_cast<SegMeta<SEG>*>(smem + 2 * 16 * SEG * 16 + kSegFloats * sizeof(float));
    const int warp = threadIdx.x >> 5;
    const Frag f;
    uint32_t DAh[4], DAl[4], DTh[2][2], DTl[2][2];
    frag_a<P>(kSetSenseA, DAh, DAl);
    frag_b<P>(kSetSenseB, DTh, DTl);
    int rk[2][4];   // ranks of R[g + 8 (i>>1)][2q + (i&1) + 8 nt] = C[u = 2q + (i&1) + 8 nt][v = g + 8 (i>>1)]
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) rk[nt][i] = zz_rank(2 * f.q + (i & 1) + 8 * nt, f.g + 8 * (i >> 1), 16);

    const ImgGeom& g = a.g;
    const bool vec = ((reinterpret_cast<uintptr_t>(a.img) | (uintptr_t)g.pitch |
                       (uintptr_t)(g.n_img > 1 ? g.img_stride : 0)) & 15) == 0;
    int64_t r0, r1;
    cta_range(ntot, &r0, &r1);
    const int nseg = (int)((r1 - r0 + SEG - 1) / SEG);
    if (nseg <= 0) return;
    griddep_wait();
    MetaRaw raw;
    if (warp == 0) {
        sense_meta_store(seg_geom<SEG>(r0, r1, 0), sense_meta_load(a, seg_geom<SEG>(r0, r1, 0)), meta[0]);
        if (1 < nseg) raw = sense_meta_load(a, seg_geom<SEG>(r0, r1, 1));
    }
    __syncthreads();
    sense_pixels(a, meta[0], pix[0], vec);
    cp_async_commit();
    int mi = 0;
    for (int j = 0; j < nseg; ++j) {
        const int mn = mi == 2 ? 0 : mi + 1;
        if (j + 1 < nseg && warp == 0) {
            sense_meta_store(seg_geom<SEG>(r0, r1, j + 1), raw, meta[mn]);
            if (j + 2 < nseg) raw = sense_meta_load(a, seg_geom<SEG>(r0, r1, j + 2));
        }
        cp_async_wait_all();
        __syncthreads();
        if (j + 1 < nseg) sense_pixels(a, meta[mn], pix[(j + 1) & 1], vec);
        cp_async_commit();

        const SegMeta<SEG>& M = meta[mi];
        const int nblk = M.sg.nblk;
        const uint8_t* px = pix[j & 1];
        float* os = ost + M.sh;
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
            const int m = M.cnt[c];
            float* ob = os + M.rel[c];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (rk[nt][i] < m) ob[rk[nt][i]] = R[nt][i];
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
        mi = mn;
    }
    cp_async_wait_all();
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
cudaError_t launch_recon_tc_p(const ReconArgs& a, cudaStream_t s) {
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
}  // namespace

cudaError_t setup_tc_fragments() {
    tc_frag_setup_kernel<<<1, 32>>>();
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
