// IDA (Sec. VI): the linear part of one iteration (Eqs. 25, 28 and the
// residual norm of Eq. 15) and the plain denoiser D_sigma.
#include "abcs_common.cuh"

namespace abcs {
ABCS_TU_TABLES(ida)
}  // namespace abcs

#include "dct_tile.cuh"
#include "tc_frag.cuh"

namespace abcs {

namespace {

// ---------------------------------------------------------------------------
// Linear step, fused per block:  c = DCT(x);  for the measured ranks
//   z = y - c + z_prev / D_F           (Eq. 25 + Onsager term alpha = 1/D_F, Eq. 28)
//   c <- c + z                          (adds A^T z in the DCT domain)
// then r = IDCT(c) = x + A^T z, and the CTA's share of ||z||^2 in FP64.
// ---------------------------------------------------------------------------
// One tile: NB = 256 / B blocks of one block row.  All pointers address the
// tile's first block / pixel; coefficient indices are coeff_base +
// offsets[.].  Returns the tile's ||z||^2 (valid in thread 0).
struct LinTile {
    const int32_t* counts;
    const int64_t* offsets;
    int64_t coeff_base;
    const float* y;
    const float* x;        // NULL: x = 0
    const float* z_prev;   // NULL: z_prev = 0
    float* z;
    float* r;
    int64_t pix;           // pixel index of the tile's top-left pixel in x / r
    int Wc;                // row stride of x / r
    int nblk;
    float inv_df;
    uint32_t* status;
};

// ZP_STAGE: z_prev staged in shared memory beside y (two staging buffers);
// otherwise it is read from global memory where it is used (one buffer).
template <int B, bool ZP_STAGE = true>
ABCS_D double linear_tile(const LinTile& L, unsigned char* smem, int* rel, int64_t* s_start, double* shd) {
    using Tl = Tile<B>;
    const TileSmem<B> sm(smem, ZP_STAGE ? 2 : 1);
    float* Ts = sm.Ts;
    float* Ys = sm.P[0];       // y, overwritten in place by z
    float* Zp = sm.P[1];       // z_prev (ZP_STAGE)
    uint16_t* rk = sm.rk;
    const int t = threadIdx.x, nblk = L.nblk;
    __syncthreads();           // smem of a previous tile is free
    load_rank_table<B>(rk);
    if (t < 32) {
        if (t == 0) *s_start = L.coeff_base + L.offsets[0];
        tile_prefix<B>(L.counts, nblk, rel, L.status);
    }
    __syncthreads();
    const int64_t start = *s_start;
    const int n_in = rel[nblk];
    stage_in_async(Ys, L.y, start, n_in);
    if (ZP_STAGE && L.z_prev) stage_in_async(Zp, L.z_prev, start, n_in);
    cp_async_commit();

    const int b = t / B, n = t % B;
    const int64_t o = L.pix + (int64_t)n * L.Wc + b * B;
    {
        float x[B];
        if (L.x && b < nblk) {
            load_f32_row<B>(L.x + o, aligned16(L.x + o), x);
        } else {
#pragma unroll
            for (int i = 0; i < B; ++i) x[i] = 0.f;
        }
        fwd_rows_to_smem<B>(x, Ts);
    }
    cp_async_wait_all();
    __syncthreads();

    // column mapping: forward DCT, residual update of the measured
    // coefficients, inverse DCT -- all in registers.  ||z||^2: each thread
    // sums its (at most B) terms in FP32, the CTA sum is an FP32 tree (this
    // GPU's FP64 pipe is narrow); the tile's partial is stored in FP64.
    float nz = 0.f;
    {
        const int v = t % B;
        float* col = Ts + b * Tl::BLK + v;
        float x[B], c[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = col[i * Tl::LD];
        fdct<B>(x, c);
        const int sh = (int)(start & 3);
        const int r0 = rel[min(b, nblk)], m = (b < nblk) ? rel[b + 1] - r0 : 0;
        float* ys = Ys + sh + r0;
        const float* zs = ZP_STAGE ? Zp + sh + r0 : (L.z_prev ? L.z_prev + start + r0 : nullptr);
        const bool has_zp = L.z_prev != nullptr;
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int r = rk[u * B + v];
            if (r < m) {
                const float zp = has_zp ? zs[r] : 0.f;
                const float z = (ys[r] - c[u]) + zp * L.inv_df;
                ys[r] = z;
                c[u] += z;
                nz = fmaf(z, z, nz);
            }
        }
        idct<B>(c, x);
#pragma unroll
        for (int i = 0; i < B; ++i) col[i * Tl::LD] = x[i];
    }
    __syncthreads();
    if (b < nblk) {
        float x[B];
        inv_rows_from_smem<B>(Ts, x);
        store_f32_row<B>(L.r + o, aligned16(L.r + o), x);
    }
    stage_out(Ys, L.z, start, n_in);
    return (double)block_sum(nz, reinterpret_cast<float*>(shd));
}

template <int B>
__global__ void __launch_bounds__(256, (B == 16 ? 3 : 4)) ida_linear_kernel(IdaLinArgs a) {
    using Tl = Tile<B>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int rel[Tl::NB + 1];
    __shared__ int64_t s_start;
    __shared__ double shd[32];
    const ImgGeom& g = a.g;
    const int k = blockIdx.z, bi = blockIdx.y, bj0 = blockIdx.x * Tl::NB;
    const int64_t gi0 = (int64_t)k * g.n_blocks + (int64_t)bi * g.nbw + bj0;
    LinTile L;
    L.counts = a.counts + gi0;
    L.offsets = a.offsets + gi0;
    L.coeff_base = 0;
    L.y = a.y; L.x = a.x; L.z_prev = a.z_prev; L.z = a.z; L.r = a.r;
    L.pix = (int64_t)k * g.Hc * g.Wc + (int64_t)(bi * B) * g.Wc + bj0 * B;
    L.Wc = g.Wc;
    L.nblk = min(Tl::NB, g.nbw - bj0);
    L.status = a.status;
    griddep_wait();
    L.inv_df = a.alpha ? a.alpha[k] : a.inv_df;
    const double nz = linear_tile<B>(L, smem, rel, &s_start, shd);
    if (threadIdx.x == 0)
        a.partial[(int64_t)k * gridDim.x * gridDim.y + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = nz;
}

template <int B>
static cudaError_t launch_lin_B(const IdaLinArgs& a, cudaStream_t s) {
    using Tl = Tile<B>;
    const size_t smem = Tl::smem_bytes(2);
    cudaError_t e = cudaFuncSetAttribute(ida_linear_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((a.g.nbw + Tl::NB - 1) / Tl::NB), (unsigned)a.g.nbh, (unsigned)a.g.n_img);
    return launch_pdl(ida_linear_kernel<B>, grid, dim3(256), smem, s, a);
}

// ---------------------------------------------------------------------------
// Linear step on the tensor cores (B = 16, the tensor-core precisions).  One
// warp keeps a 16 x 16 block in mma.sync fragments through
//   forward   V = D X^T, then R = V D^T = C^T          (A = D, then A = V)
//   residual  z = y - c + z_prev / D_F on the measured ranks (Eqs. 25, 28)
//   adjoint   X_z = D^T Z D of the masked residual Z    (A = D^T, then A = Y)
//   r = x + X_z
// Lane (g, q) holds pixel rows g, g + 8 x columns 2q, 2q + 1, 2q + 8, 2q + 9:
// the B-operand layout of X^T and the accumulator layout of X_z alike, so x
// stays in registers from its load to the final addition, and the forward's
// accumulators hold exactly the coefficients that the adjoint's B operand
// needs in the same lane.  Adding the transformed correction to x (rather
// than inverting c + z) keeps x's components outside the measured ranks
// exact.  The B operands of D^T and D are the A operands of D and D^T in
// another register order (b[nt][j] = a[nt + 2 j]), so two constant
// fragments serve all four products.
// ---------------------------------------------------------------------------
__device__ uint32_t g_ida_frag[3][2][8][32];   // [precision][A of D, A of D^T][hi 0-3, lo 4-7][lane]

template <int P>
ABCS_D void ida_frag_setup_p() {
    const int lane = threadIdx.x & 31;
    uint32_t h[4], l[4];
    for (int s = 0; s < 2; ++s) {
        load_a_const<P>(s == 1, h, l);
        for (int i = 0; i < 4; ++i) {
            g_ida_frag[pidx<P>()][s][i][lane] = h[i];
            g_ida_frag[pidx<P>()][s][4 + i][lane] = l[i];
        }
    }
}

__global__ void ida_frag_setup_kernel() {
    ida_frag_setup_p<kP16>();
    ida_frag_setup_p<kPB16>();
    ida_frag_setup_p<kPB1>();
}

// *p = v if r < m
ABCS_D void st_global_lt(float* p, float v, int r, int m) {
    asm volatile("{\n .reg .pred q;\n setp.lt.s32 q, %2, %3;\n @q st.global.f32 [%0], %1;\n}\n" ::"l"(p),
                 "f"(v), "r"(r), "r"(m)
                 : "memory");
}

constexpr int kTcNB = 16;                       // blocks of a tile (one block row, 256 pixel columns)
// Coefficient staging buffers hold up to kTcCap coefficients (160 per block
// on average, subrate 0.625); a tile with more reads y and z_prev from
// global memory instead.  The cap keeps three CTAs resident per SM.
constexpr int kTcCap = 2560;
constexpr int kTcStage = kTcCap + 4;            // floats of a packed coefficient staging buffer
constexpr int kTcX = kTcNB * 256;               // floats of a tile's x stage
// dynamic shared memory: two stages of (x, y, z_prev), three metadata slots
struct TcMeta {
    int64_t start;     // index of the tile's first coefficient
    int64_t pix;       // pixel index of the tile's top-left pixel
    int rel[kTcNB + 1];
    int nblk;
    int k;             // image
};
constexpr size_t kTcStageBytes = (size_t)(kTcX + 2 * kTcStage) * 4;
constexpr size_t kTcSmem = 2 * kTcStageBytes + 3 * sizeof(TcMeta);

// A tile's counts and first offset, loaded by warp 0 two tiles ahead:
// lane l holds the counts of blocks 2l and 2l + 1.
struct TcRaw {
    int c0, c1;
    int64_t start;
};

struct TcTile {
    int k, by, bx, nblk;
    int64_t gi0;       // first block of the tile in counts / offsets
};

// tile j (< 2^31) -> image, block row, tile column
ABCS_D TcTile tc_tile(const ImgGeom& g, int ntx, int j) {
    TcTile t;
    const int per_img = ntx * g.nbh;
    t.k = j / per_img;
    const int r = j - t.k * per_img;
    t.by = r / ntx;
    t.bx = r - t.by * ntx;
    t.nblk = min(kTcNB, g.nbw - t.bx * kTcNB);
    t.gi0 = (int64_t)t.k * g.n_blocks + (int64_t)t.by * g.nbw + t.bx * kTcNB;
    return t;
}

ABCS_D TcRaw tc_raw_load(const IdaLinArgs& a, const TcTile& t) {
    const int lane = threadIdx.x & 31;
    TcRaw r;
    r.c0 = 2 * lane < t.nblk ? __ldg(a.counts + t.gi0 + 2 * lane) : 0;
    r.c1 = 2 * lane + 1 < t.nblk ? __ldg(a.counts + t.gi0 + 2 * lane + 1) : 0;
    r.start = lane == 0 ? __ldg(a.offsets + t.gi0) : 0;
    return r;
}

// warp 0: counts clamped to [0, 256] (a clamp sets ABCS_DEV_BADCOUNT), block
// offsets relative to the tile's first coefficient
ABCS_D void tc_meta_store(const IdaLinArgs& a, const TcTile& t, TcRaw r, TcMeta& M) {
    const int lane = threadIdx.x & 31;
    bool bad = false;
    if (r.c0 < 0 || r.c0 > 256) { bad = true; r.c0 = r.c0 < 0 ? 0 : 256; }
    if (r.c1 < 0 || r.c1 > 256) { bad = true; r.c1 = r.c1 < 0 ? 0 : 256; }
    const int pair = r.c0 + r.c1;
    int incl = pair;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    const int excl = incl - pair;
    if (2 * lane < t.nblk) M.rel[2 * lane] = excl;
    if (2 * lane + 1 < t.nblk) M.rel[2 * lane + 1] = excl + r.c0;
    const int64_t start = __shfl_sync(0xffffffffu, r.start, 0);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane == 0) {
        M.rel[t.nblk] = total;
        M.start = start;
        M.nblk = t.nblk;
        M.k = t.k;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(a.status, ABCS_DEV_BADCOUNT);
}

// x chunk (block c, pixel row r, 16-byte chunk h) at float offset
// 256 c + 16 r + 4 (h ^ s(r)), s(r) = 2 ((r >> 1) & 1): the fragment loads
// (lane (g, q): rows g, g + 8, float pairs 2q, 2q + 8) are then free of
// bank conflicts
ABCS_D int tc_xoff(int c, int r, int h) { return 256 * c + 16 * r + 4 * (h ^ (((r >> 1) & 1) << 1)); }

// all threads: x of the tile (16-byte copies; x and Wc 16-byte aligned),
// y and z_prev ranges
ABCS_D void tc_stage_in(const IdaLinArgs& a, const ImgGeom& g, const TcMeta& M, float* xs, float* ys, float* zs) {
    if (a.x) {
        // thread (row r0, block c, chunk h) copies rows r0 + 4 i (i < 4): the
        // swizzle term of rows r0 + 4 i is that of r0, so they sit 64 i floats on
        const int h = threadIdx.x & 3, c = (threadIdx.x >> 2) & 15, r0 = threadIdx.x >> 6;
        if (c < M.nblk) {
            const float* src = a.x + M.pix + (int64_t)r0 * g.Wc + 16 * c + 4 * h;
            float* dst = xs + tc_xoff(c, r0, h);
            const int64_t step = 4 * (int64_t)g.Wc;
#pragma unroll
            for (int i = 0; i < 4; ++i) cp_async16(dst + 64 * i, src + i * step);
        }
    }
    const int n = M.rel[M.nblk];
    if (n <= kTcCap) {
        if (a.z_prev) stage_in_async2(ys, a.y, zs, a.z_prev, M.start, n);
        else stage_in_async(ys, a.y, M.start, n);
    }
}

// Lane constants of the transform, computed once per thread.
struct TcLane {
    uint32_t xo[2][2];     // byte offset in a block's x stage of rows g + 8 h, columns 2q + 8 p, + 1
    uint32_t rk[2];        // ranks of R[nt][i] = C[2q + (i & 1) + 8 nt][g + 8 (i >> 1)], byte 4 nt + i
    int ro;                // pixel offset of row g, column 2q in a block (row stride Wc)
};

ABCS_D int tc_rank(const TcLane& L, int nt, int i) { return (int)((L.rk[nt] >> (8 * i)) & 0xFFu); }


// One 16 x 16 block by one warp.  xb: shared address of its x stage
// (tc_xoff layout, block 0); yb: shared address of its first staged
// coefficient, z_prev zoff bytes further (STAGED), or yg / zpg: the same
// coefficients in global memory; zg: its z; rb: r at its top-left pixel plus
// the lane offset ro, rows 8 apart at rb8.  Returns the lane's FP32 sum of
// z^2 (at most 8 terms).
template <int P, bool STAGED, bool FULL>
ABCS_D float tc_block(uint32_t xb, uint32_t yb, uint32_t zoff, const float* yg, const float* zpg, float* zg,
                      float* rb, float* rb8, int m, float inv_df, bool has_x_, bool has_zp_, const uint32_t (&Dh)[4],
                      const uint32_t (&Dl)[4], const uint32_t (&Th)[4], const uint32_t (&Tl)[4], const TcLane& ln) {
    // FULL: x and z_prev are both given (every iteration after the first),
    // known at compile time so no per-coefficient test remains
    const bool has_x = FULL || has_x_, has_zp = FULL || has_zp_;
    float R[2][4] = {};
    if (has_x) {
        float V[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const float2 x0 = lds_f2(xb + ln.xo[nt][0]), x1 = lds_f2(xb + ln.xo[nt][1]);
            uint32_t bh0, bl0, bh1, bl1;
            split2<P>(x0.x, x0.y, bh0, bl0);
            split2<P>(x1.x, x1.y, bh1, bl1);
            mma_split<P>(V[nt], Dh, Dl, bh0, bh1, bl0, bl1);
        }
        uint32_t Ah[4], Al[4];
        split2<P>(V[0][0], V[0][1], Ah[0], Al[0]);
        split2<P>(V[0][2], V[0][3], Ah[1], Al[1]);
        split2<P>(V[1][0], V[1][1], Ah[2], Al[2]);
        split2<P>(V[1][2], V[1][3], Ah[3], Al[3]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_split<P>(R[nt], Ah, Al, Dh[nt], Dh[nt + 2], Dl[nt], Dl[nt + 2]);
    }
    float nz = 0.f;
    float Z[2][4];
    // staged: every lane reads in-range stage words (index 0 where the rank
    // is not measured); from global memory only measured ranks are read; z
    // is stored under a predicate
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = tc_rank(ln, nt, i);
            const bool v = r < m;
            float yv, zp;
            if (STAGED) {
                const uint32_t ad = yb + 4u * (uint32_t)(v ? r : 0);
                yv = lds_f(ad);
                zp = has_zp ? lds_f(ad + zoff) : 0.f;
            } else {
                yv = v ? yg[r] : 0.f;
                zp = (has_zp && v) ? zpg[r] : 0.f;
            }
            const float z = v ? (yv - R[nt][i]) + zp * inv_df : 0.f;
            st_global_lt(zg + r, z, r, m);
            nz = fmaf(z, z, nz);
            Z[nt][i] = z;
        }
    float Y[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        uint32_t bh0, bl0, bh1, bl1;
        split2<P>(Z[0][2 * nt], Z[0][2 * nt + 1], bh0, bl0);
        split2<P>(Z[1][2 * nt], Z[1][2 * nt + 1], bh1, bl1);
        mma_split<P>(Y[nt], Th, Tl, bh0, bh1, bl0, bl1);
    }
    uint32_t Ah[4], Al[4];
    split2<P>(Y[0][0], Y[0][1], Ah[0], Al[0]);
    split2<P>(Y[0][2], Y[0][3], Ah[1], Al[1]);
    split2<P>(Y[1][0], Y[1][1], Ah[2], Al[2]);
    split2<P>(Y[1][2], Y[1][3], Ah[3], Al[3]);
    float X[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) mma_split<P>(X[nt], Ah, Al, Th[nt], Th[nt + 2], Tl[nt], Tl[nt + 2]);
    // r = x + X_z; X[p][i]: pixel row g + 8 (i >> 1), column 2q + (i & 1) + 8 p
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 xv = has_x ? lds_f2(xb + ln.xo[h][p]) : make_float2(0.f, 0.f);
            *reinterpret_cast<float2*>((h ? rb8 : rb) + 8 * p) =
                make_float2(xv.x + X[p][2 * h], xv.y + X[p][2 * h + 1]);
        }
    return nz;
}

// One tile from the stage, 8 warps: warp w transforms blocks w and w + 8.
// xs, ys: shared addresses of the stage's x and y buffers (z_prev follows y
// at kTcStage floats).  Returns the lane's FP32 sum of z^2 (at most 16 terms).
template <int P, bool STAGED, bool FULL>
ABCS_D float tc_transform(const IdaLinArgs& a, const ImgGeom& g, const TcMeta& M, uint32_t xs, uint32_t ys,
                          float inv_df, const uint32_t (&Dh)[4], const uint32_t (&Dl)[4], const uint32_t (&Th)[4],
                          const uint32_t (&Tl)[4], const TcLane& ln) {
    const int warp = threadIdx.x >> 5;
    const uint32_t sh = (uint32_t)(M.start & 3);
    float nz = 0.f;
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
        const int c = warp + 8 * j;
        if (c >= M.nblk) break;
        const int r0 = M.rel[c], m = M.rel[c + 1] - r0;
        float* rb = a.r + M.pix + c * 16 + ln.ro;
        nz += tc_block<P, STAGED, FULL>(xs + 1024u * (uint32_t)c, ys + 4u * (sh + (uint32_t)r0), 4u * kTcStage,
                                  a.y + M.start + r0, a.z_prev + M.start + r0, a.z + M.start + r0, rb,
                                  rb + 8 * (int64_t)g.Wc, m, inv_df, a.x != nullptr, a.z_prev != nullptr, Dh, Dl,
                                  Th, Tl, ln);
    }
    return nz;
}

// Persistent CTAs walk the tiles j = blockIdx.x, + gridDim.x, ...; tile
// j + G's x, y and z_prev are copied (cp.async) while tile j is
// transformed, and warp 0 loads tile j + 2G's counts.  One barrier per
// tile.  Tile j's ||z||^2 goes to partial[j] (the same slot as the per-tile
// kernel's) in FP64: each warp sums its lanes in FP32 (at most 512 terms),
// and thread 0 adds the 8 warp sums in FP32 after the next tile's barrier
// (FP64 adds there held warp 0 back and the other warps at the barrier).
// FULL: launched when x and z_prev are both given (every iteration after the
// first), so the block transform tests neither.
template <int P, bool FULL>
__global__ void __launch_bounds__(256, 3) ida_linear_tc_kernel(IdaLinArgs a, int ntx, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float swarp[2][8];
    TcMeta* meta = reinterpret_cast<TcMeta*>(smem + 2 * kTcStageBytes);
    auto xs = [&](int b) { return reinterpret_cast<float*>(smem + b * kTcStageBytes); };
    auto ys = [&](int b) { return xs(b) + kTcX; };
    auto zs = [&](int b) { return xs(b) + kTcX + kTcStage; };
    const ImgGeom& g = a.g;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Frag f;
    uint32_t Dh[4], Dl[4], Th[4], Tl[4];
    {
        const uint32_t* tb = &g_ida_frag[pidx<P>()][0][0][lane];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            Dh[i] = tb[32 * i];
            Dl[i] = tb[32 * (4 + i)];
            Th[i] = tb[256 + 32 * i];
            Tl[i] = tb[256 + 32 * (4 + i)];
        }
    }
    TcLane ln;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        uint32_t w = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            w |= (uint32_t)zz_rank(2 * f.q + (i & 1) + 8 * nt, f.g + 8 * (i >> 1), 16) << (8 * i);
        ln.rk[nt] = w;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int p = 0; p < 2; ++p)
            ln.xo[h][p] = 4u * (uint32_t)(tc_xoff(0, f.g + 8 * h, (f.q >> 1) + 2 * p) + 2 * (f.q & 1));
    ln.ro = f.g * a.g.Wc + 2 * f.q;
    const int G = gridDim.x;
    const int j0 = blockIdx.x;
    if (j0 >= ntiles) return;
    griddep_wait();
    auto tile_pix = [&](const TcTile& t) {
        return (int64_t)t.k * g.Hc * g.Wc + (int64_t)(t.by * 16) * g.Wc + t.bx * 256;
    };
    TcRaw raw;
    if (warp == 0) {
        const TcTile t0 = tc_tile(g, ntx, j0);
        tc_meta_store(a, t0, tc_raw_load(a, t0), meta[0]);
        if (lane == 0) meta[0].pix = tile_pix(t0);
        if (j0 + G < ntiles) raw = tc_raw_load(a, tc_tile(g, ntx, j0 + G));
    }
    __syncthreads();
    tc_stage_in(a, g, meta[0], xs(0), ys(0), zs(0));
    cp_async_commit();
    int i = 0;
    for (int j = j0; j < ntiles; j += G, ++i) {
        const int b = i & 1, mi = i % 3, mn = (i + 1) % 3;
        const bool next = j + G < ntiles;
        if (warp == 0 && next) {
            const TcTile tn = tc_tile(g, ntx, j + G);
            tc_meta_store(a, tn, raw, meta[mn]);
            if (lane == 0) meta[mn].pix = tile_pix(tn);
            if (j + 2 * G < ntiles) raw = tc_raw_load(a, tc_tile(g, ntx, j + 2 * G));
        }
        cp_async_wait_all();          // tile j's stage has landed (this thread's copies)
        __syncthreads();              // ... everyone's; meta[mn] written; stage b ^ 1 free; swarp[b ^ 1] final
        if (threadIdx.x == 0 && i > 0) {
            float sum = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) sum += swarp[b ^ 1][w];
            a.partial[j - G] = (double)sum;
        }
        if (next) tc_stage_in(a, g, meta[mn], xs(b ^ 1), ys(b ^ 1), zs(b ^ 1));
        cp_async_commit();
        const TcMeta& M = meta[mi];
        const float inv_df = a.alpha ? __ldg(a.alpha + M.k) : a.inv_df;
        const uint32_t xsa = (uint32_t)__cvta_generic_to_shared(xs(b)), ysa = (uint32_t)__cvta_generic_to_shared(ys(b));
        const float nz = warp_sum(M.rel[M.nblk] <= kTcCap
                                      ? tc_transform<P, true, FULL>(a, g, M, xsa, ysa, inv_df, Dh, Dl, Th, Tl, ln)
                                      : tc_transform<P, false, FULL>(a, g, M, xsa, ysa, inv_df, Dh, Dl, Th, Tl, ln));
        if (lane == 0) swarp[b][warp] = nz;
    }
    cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int b = (i - 1) & 1;
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) sum += swarp[b][w];
        a.partial[j0 + (i - 1) * G] = (double)sum;
    }
}

template <int P, bool FULL>
static cudaError_t launch_lin_tc_k(const IdaLinArgs& a, cudaStream_t s) {
    const int ntx = (a.g.nbw + kTcNB - 1) / kTcNB;
    const int64_t ntiles = (int64_t)ntx * a.g.nbh * a.g.n_img;
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    int dev, sms, per_sm;
    cudaError_t e = cudaFuncSetAttribute(ida_linear_tc_kernel<P, FULL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmem);
    if (!e) e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ida_linear_tc_kernel<P, FULL>, 256, kTcSmem);
    if (e) return e;
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    return launch_pdl(ida_linear_tc_kernel<P, FULL>, dim3(grid), dim3(256), kTcSmem, s, a, ntx, (int)ntiles);
}

template <int P>
static cudaError_t launch_lin_tc(const IdaLinArgs& a, cudaStream_t s) {
    return a.x && a.z_prev ? launch_lin_tc_k<P, true>(a, s) : launch_lin_tc_k<P, false>(a, s);
}

// sigma^t = sqrt(||z^t||^2 / m) per image (Eq. 15); m = the image's
// measurement count.  Partials are summed in a fixed order.
__global__ void ida_sigma_kernel(const double* __restrict__ partial, int cpi,
                                 const int64_t* __restrict__ offsets, int64_t nB,
                                 float* __restrict__ sigma, float* __restrict__ trace, int iters,
                                 int t, uint32_t* status) {
    griddep_wait();
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < cpi; j += 32) s += partial[(int64_t)k * cpi + j];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        // the FP64 sum rounded once to FP32, then an FP32 division and square
        // root (a few ulp; this GPU's FP64 divide and square root are slow)
        const int64_t m = offsets[(int64_t)(k + 1) * nB] - offsets[(int64_t)k * nB];
        const float v = m > 0 ? sqrtf((float)s / (float)m) : 0.f;
        if (!isfinite(v)) set_status(status, ABCS_DEV_NONFINITE);
        sigma[k] = v;
        if (trace) trace[(int64_t)k * iters + t] = v;
    }
}

// ---------------------------------------------------------------------------
// D-AMP / DAMP-D (Eqs. 24, 27): the Onsager coefficient from a Monte-Carlo
// estimate of the denoiser's divergence, div ~ b^T (D(r + eps b) - D(r)) / eps
// with eps = eps_rel max|r| per image and the caller's probe b.
// Grid (chunks, images) for the element-wise kernels.
// ---------------------------------------------------------------------------
constexpr int kDampThreads = 256;

// amax[k] = bits of max |r| over image k (non-negative floats order as
// unsigned integers); cleared by damp_clear_kernel first
__global__ void damp_clear_kernel(unsigned* __restrict__ amax) {
    griddep_wait();
    amax[blockIdx.x] = 0u;
}

__global__ void __launch_bounds__(kDampThreads) damp_amax_kernel(const float* __restrict__ r, int64_t per_img,
                                                                 unsigned* __restrict__ amax) {
    griddep_wait();
    const int k = blockIdx.y;
    const float* rk = r + (int64_t)k * per_img;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(rk[i]));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax + k, __float_as_uint(m));
}

ABCS_D float damp_eps(unsigned amax_bits, float eps_rel) {
    const float e = eps_rel * __uint_as_float(amax_bits);
    return e > 0.f ? e : eps_rel;
}

__global__ void __launch_bounds__(kDampThreads) damp_perturb_kernel(const float* __restrict__ r,
                                                                    const float* __restrict__ probe, int64_t per_img,
                                                                    const unsigned* __restrict__ amax, float eps_rel,
                                                                    float* __restrict__ rp) {
    griddep_wait();
    const int k = blockIdx.y;
    const float eps = damp_eps(amax[k], eps_rel);
    const int64_t o = (int64_t)k * per_img;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        rp[o + i] = fmaf(eps, __ldg(probe + o + i), r[o + i]);
}

// per CTA: sum of b (xp - x) in FP64
__global__ void __launch_bounds__(kDampThreads) damp_div_kernel(const float* __restrict__ probe,
                                                                const float* __restrict__ xp,
                                                                const float* __restrict__ x, int64_t per_img,
                                                                double* __restrict__ partial) {
    __shared__ double sh[32];
    griddep_wait();
    const int k = blockIdx.y;
    const int64_t o = (int64_t)k * per_img;
    float a = 0.f;                                  // a thread's few terms in FP32, the CTA sum in FP64
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += (int64_t)gridDim.x * blockDim.x)
        a = fmaf(__ldg(probe + o + i), xp[o + i] - x[o + i], a);
    const double acc = block_sum((double)a, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = acc;
}

// one warp per image: partials in a fixed order, alpha = inv_df div / M
__global__ void damp_alpha_kernel(const double* __restrict__ partial, int chunks, const int64_t* __restrict__ offsets,
                                  int64_t nB, const unsigned* __restrict__ amax, float eps_rel, float inv_df,
                                  float* __restrict__ alpha, float* __restrict__ trace, int iters, int t,
                                  uint32_t* status) {
    griddep_wait();
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < chunks; j += 32) s += partial[(int64_t)k * chunks + j];
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        const int64_t m = offsets[(int64_t)(k + 1) * nB] - offsets[(int64_t)k * nB];
        const double div = s / (double)damp_eps(amax[k], eps_rel);
        const double v = m > 0 ? (double)inv_df * div / (double)m : 0.0;
        if (!isfinite(v)) set_status(status, ABCS_DEV_NONFINITE);
        alpha[k] = (float)v;
        if (trace) trace[(int64_t)k * iters + t + 1] = (float)v;
    }
}

// ---------------------------------------------------------------------------
// Plain denoiser: translation-invariant 8x8 DCT hard thresholding.  Every
// pixel is the mean, over the 64 8x8 windows that contain it, of the window
// after an orthonormal DCT, zeroing of the AC coefficients with
// |c| <= lambda sigma, and the inverse DCT.  Outside the image the input is
// extended half-sample symmetrically.
//
// A CTA produces a 240 x 64 output tile.  It walks the window rows wy from
// y0-7 to y0+63; per window row:
//   (a) column DCT of 8 input rows, shared by all windows of the row
//       (thread per input column, sliding 8-row register window);
//   (b) thread per window: row DCT, threshold, row inverse -> Q (smem);
//   (c) thread per output column: overlap-add of the 8 windows covering it
//       and the column inverse, accumulated in 8 sliding registers; the top
//       row is complete and written out.
// (b) and (c) run twice per window row, on frequency rows 0-3 and then 4-7.
// Steps (b) and (c) carry the frequency rows u in pairs (2p, 2p + 1) through
// packed FP32x2 arithmetic (one instruction, two FP32 operations, each
// rounded as the scalar one), so the results are those of the scalar
// transforms.  Every output accumulates in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kTW = 240, kWin = kTW + 7, kCols = kTW + 14, kQS2 = 17;
// Vs: [4 row pairs][256 columns] float2; Qs: [kWin windows][kQS2] float2 for
// one half of the row pairs at a time (16 used: 2 row pairs x 8 positions;
// 17 keeps the per-window rows on distinct bank pairs).  Halving Q keeps the
// CTA at 42 KB, five CTAs per SM.
constexpr size_t kTidctSmem = (4 * 256 + kWin * kQS2) * sizeof(float2);

ABCS_D int reflect(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;           // inside: no division
    const int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i < n ? i : p - 1 - i;
}

ABCS_D float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
ABCS_D float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }   // exact a - b
ABCS_D float2 f2_fma(float c, float2 x, float2 acc) { return __ffma2_rn(make_float2(c, c), x, acc); }
ABCS_D float2 f2_mul(float c, float2 x) { return __fmul2_rn(make_float2(c, c), x); }

// fdct_rec / idct_rec on two vectors at once, the same operations in the
// same order per component
template <int S, int N>
ABCS_D void fdct8x2_rec(const float2* x, float2* c) {
    if constexpr (N == 1) {
        c[0] = f2_mul(Dc<8>(0, 0), x[0]);
    } else {
        constexpr int H = N / 2;
        float2 sm[H], d[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
            sm[n] = f2_add(x[n], x[N - 1 - n]);
            d[n] = f2_sub(x[n], x[N - 1 - n]);
        }
        fdct8x2_rec<2 * S, H>(sm, c);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int n = 0; n < H; ++n) acc = f2_fma(Dc<8>(S * (2 * j + 1), n), d[n], acc);
            c[S * (2 * j + 1)] = acc;
        }
    }
}

template <int S, int N>
ABCS_D void idct8x2_rec(const float2* c, float2* x) {
    if constexpr (N == 2) {
        // the DC product D[0][0] c[0] enters both sums unrounded (one FMA
        // each), as the scalar transform is compiled
        const float2 o = f2_fma(Dc<8>(S, 0), c[S], make_float2(0.f, 0.f));
        const float d0 = Dc<8>(0, 0);
        x[0] = __ffma2_rn(make_float2(d0, d0), c[0], o);
        x[1] = __ffma2_rn(make_float2(d0, d0), c[0], make_float2(-o.x, -o.y));
    } else if constexpr (N == 1) {
        x[0] = f2_mul(Dc<8>(0, 0), c[0]);
    } else {
        constexpr int H = N / 2;
        float2 e[H];
        idct8x2_rec<2 * S, H>(c, e);
#pragma unroll
        for (int n = 0; n < H; ++n) {
            float2 o = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < H; ++j) o = f2_fma(Dc<8>(S * (2 * j + 1), n), c[S * (2 * j + 1)], o);
            x[n] = f2_add(e[n], o);
            x[N - 1 - n] = f2_sub(e[n], o);
        }
    }
}

// One 240 x TH output tile of the plain denoiser (img, dst: one image).
template <int TH>
ABCS_D void tidct_tile(const float* __restrict__ img, float* __restrict__ dst, int H, int W, int x0, int y0,
                       float thr, unsigned char* smem) {
    float2* Vs = reinterpret_cast<float2*>(smem);     // [4][256]
    float2* Qs = Vs + 4 * 256;                         // [kWin][kQS2]
    const int t = threadIdx.x;
    __syncthreads();                                   // smem of a previous tile is free

    // (a) state: this thread's input column and its 8-row window
    const bool has_col = t < kCols;
    const int xc = reflect(x0 - 7 + t, W);
    float col[8];
    if (has_col) {
#pragma unroll
        for (int i = 0; i < 8; ++i) col[i] = __ldg(img + (int64_t)reflect(y0 - 7 + i, H) * W + xc);
    }
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
    const int ylast = min(y0 + TH, H);

    for (int wy = y0 - 7; wy < ylast; ++wy) {
        if (has_col) {
            float V[8];
            fdct<8>(col, V);
#pragma unroll
            for (int p = 0; p < 4; ++p) Vs[p * 256 + t] = make_float2(V[2 * p], V[2 * p + 1]);
#pragma unroll
            for (int i = 0; i < 7; ++i) col[i] = col[i + 1];
            if (wy + 8 < ylast + 7) col[7] = __ldg(img + (int64_t)reflect(wy + 8, H) * W + xc);
        }
        float S[8];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            __syncthreads();                           // Vs written (half 0); Q read by the last (c) (half 1)
            if (t < kWin) {
                float2* q = Qs + t * kQS2;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int p = 2 * half + pp;
                    float2 vr[8], c[8], qr[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) vr[j] = Vs[p * 256 + t + j];
                    fdct8x2_rec<1, 8>(vr, c);
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        c[v].x = (fabsf(c[v].x) > thr || (p == 0 && v == 0)) ? c[v].x : 0.f;
                        c[v].y = fabsf(c[v].y) > thr ? c[v].y : 0.f;
                    }
                    idct8x2_rec<1, 8>(c, qr);
#pragma unroll
                    for (int j = 0; j < 8; ++j) q[pp * 8 + j] = qr[j];
                }
            }
            __syncthreads();
            if (t < kTW) {
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < 8; ++d) s2 = f2_add(s2, Qs[(t + d) * kQS2 + pp * 8 + (7 - d)]);
                    S[4 * half + 2 * pp] = s2.x;
                    S[4 * half + 2 * pp + 1] = s2.y;
                }
            }
        }
        if (t < kTW) {
            float X[8];
            idct<8>(S, X);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) acc[kk] += X[kk];
            if (wy >= y0 && x0 + t < W) dst[(int64_t)wy * W + x0 + t] = acc[0] * (1.f / 64.f);
#pragma unroll
            for (int kk = 0; kk < 7; ++kk) acc[kk] = acc[kk + 1];
            acc[7] = 0.f;
        }
    }
}

template <int TH>
__global__ void __launch_bounds__(256) tidct_kernel(const float* __restrict__ in, float* __restrict__ out, int H,
                                                   int W, const float* __restrict__ sigma, float lambda) {
    extern __shared__ __align__(16) unsigned char smem[];
    griddep_wait();
    const int k = blockIdx.z;
    tidct_tile<TH>(in + (int64_t)k * H * W, out + (int64_t)k * H * W, H, W, blockIdx.x * kTW, blockIdx.y * TH,
                   lambda * __ldg(sigma + k), smem);
}

// ---------------------------------------------------------------------------
// Uneven batch: every iteration of IDA for images of different sizes and
// block sizes in ONE persistent cooperative launch.  Phases (linear step,
// per-image sigma, denoiser) are separated by grid barriers whose waits are
// bounded: a wait that exceeds `timeout` clock cycles sets
// ABCS_DEV_TIMEOUT, raises the abort flag and every CTA leaves the kernel.
// ---------------------------------------------------------------------------
#ifndef ABCS_BATCH_MINB
#define ABCS_BATCH_MINB 3
#endif

ABCS_D bool grid_sync(unsigned* bar, long long timeout, uint32_t* status, int* s_ok, bool skip_arrival = false) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile unsigned* vabort = bar + 2;
        int ok = *vabort ? 0 : 1;
        if (ok) {
            const unsigned g = *vgen;
            __threadfence();
            if (!skip_arrival && atomicAdd(bar, 1u) == gridDim.x - 1) {
                bar[0] = 0u;
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const long long t0 = clock64();
                while (*vgen == g) {
                    if (*vabort) { ok = 0; break; }
                    if (clock64() - t0 > timeout) {
                        atomicExch(bar + 2, 1u);
                        set_status(status, ABCS_DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// image owning tile `tile` (first-tile indices ascending)
ABCS_D int find_image(const BatchImg* imgs, int n, int tile, bool linear) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int f = linear ? __ldg(&imgs[mid].lin0) : __ldg(&imgs[mid].den0);
        if (f <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The phases of the persistent kernel are separate calls so that each is
// register-allocated on its own (inlined together they need 255 registers
// and spill, one CTA per SM).
// B = 32 reads z_prev from global memory: its shared memory (68.6 KB) then
// stays below the denoiser's, which keeps three CTAs per SM.
template <int B>
__device__ __noinline__ double linear_tile_call(const LinTile& L, unsigned char* smem, int* rel, int64_t* s_start,
                                                double* shd) {
    return linear_tile<B, (B < 32)>(L, smem, rel, s_start, shd);
}

template <int TH>
__device__ __noinline__ void tidct_tile_call(const float* img, float* dst, int H, int W, int x0, int y0, float thr,
                                             unsigned char* smem) {
    tidct_tile<TH>(img, dst, H, W, x0, y0, thr, smem);
}

template <int TH>
__global__ void __launch_bounds__(256, ABCS_BATCH_MINB) ida_batch_kernel(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int rel[kTileCols / 4 + 1];
    __shared__ int64_t s_start;
    __shared__ double shd[32];
    __shared__ int s_ok;
    const int G = gridDim.x;
    for (int t = 0; t < a.iters; ++t) {
        const float* xcur = t == 0 ? nullptr : (a.denoiser == ABCS_DEN_NONE ? ((t - 1) & 1 ? a.r1 : a.r0) : a.x);
        const float* zp = t == 0 ? nullptr : ((t - 1) & 1 ? a.z1 : a.z0);
        float* zc = (t & 1) ? a.z1 : a.z0;
        float* rc = (t & 1) ? a.r1 : a.r0;
        // linear step (Eqs. 25, 28) over every block row tile of every image
        for (int tile = blockIdx.x; tile < a.n_lin; tile += G) {
            const int k = find_image(a.imgs, a.n_img, tile, true);
            const BatchImg im = a.imgs[k];
            const int NB = kTileCols / im.B, tpr = (im.nbw + NB - 1) / NB;
            const int local = tile - im.lin0, bi = local / tpr, bj0 = (local - bi * tpr) * NB;
            const int64_t gi0 = im.blk0 + (int64_t)bi * im.nbw + bj0;
            LinTile L;
            L.counts = a.counts + gi0;
            L.offsets = a.offsets + gi0;
            L.coeff_base = im.coeff_base;
            L.y = a.y; L.x = xcur; L.z_prev = zp; L.z = zc; L.r = rc;
            L.pix = im.pix0 + (int64_t)(bi * im.B) * im.Wc + bj0 * im.B;
            L.Wc = im.Wc;
            L.nblk = min(NB, im.nbw - bj0);
            L.inv_df = a.inv_df;
            L.status = a.status;
            double nz = 0.0;
            switch (im.B) {
                case 4: nz = linear_tile_call<4>(L, smem, rel, &s_start, shd); break;
                case 8: nz = linear_tile_call<8>(L, smem, rel, &s_start, shd); break;
                case 16: nz = linear_tile_call<16>(L, smem, rel, &s_start, shd); break;
                default: nz = linear_tile_call<32>(L, smem, rel, &s_start, shd); break;
            }
            if (threadIdx.x == 0) a.partial[tile] = nz;
        }
        if (!grid_sync(a.bar, a.timeout, a.status, &s_ok, t == 0 && (int)blockIdx.x == a.skip_cta)) return;
        // sigma^t per image (Eq. 15), partials in a fixed order
        for (int k = blockIdx.x; k < a.n_img; k += G) {
            if (threadIdx.x < 32) {
                const BatchImg im = a.imgs[k];
                const int l1 = k + 1 < a.n_img ? a.imgs[k + 1].lin0 : a.n_lin;
                double s = 0.0;
                for (int j = im.lin0 + threadIdx.x; j < l1; j += 32) s += a.partial[j];
                s = warp_sum(s);
                if (threadIdx.x == 0) {
                    const int64_t last = im.blk0 + (int64_t)im.nbh * im.nbw - 1;
                    const int64_t m = a.offsets[last] + a.counts[last] - a.offsets[im.blk0];
                    const float v = m > 0 ? sqrtf((float)s / (float)m) : 0.f;   // as ida_sigma_kernel
                    if (!isfinite(v)) set_status(a.status, ABCS_DEV_NONFINITE);
                    a.sigma[k] = v;
                    if (a.trace) a.trace[(int64_t)k * a.iters + t] = v;
                }
            }
        }
        if (!grid_sync(a.bar, a.timeout, a.status, &s_ok)) return;
        if (a.denoiser == ABCS_DEN_TIDCT) {
            for (int tile = blockIdx.x; tile < a.n_den; tile += G) {
                const int k = find_image(a.imgs, a.n_img, tile, false);
                const BatchImg im = a.imgs[k];
                const int tx = (im.Wc + kTW - 1) / kTW;
                const int local = tile - im.den0;
                tidct_tile_call<TH>(rc + im.pix0, a.x + im.pix0, im.Hc, im.Wc, (local % tx) * kTW, (local / tx) * TH,
                                    a.lambda * a.sigma[k], smem);
            }
            if (!grid_sync(a.bar, a.timeout, a.status, &s_ok)) return;
        }
    }
}

// d[k][y][x] = m_i / B^2 of the block holding pixel (y, x) of image k; one
// image row per CTA step, B a power of two
__global__ void __launch_bounds__(256) density_kernel(ImgGeom g, const int32_t* __restrict__ counts,
                                                      float* __restrict__ out) {
    griddep_wait();
    const int rows = g.n_img * g.Hc, lb = __ffs(g.B) - 1;
    const float inv = 1.f / (float)(g.B * g.B);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = row / g.Hc, y = row - k * g.Hc;
        const int32_t* ck = counts + (int64_t)k * g.n_blocks + (int64_t)(y >> lb) * g.nbw;
        float* o = out + (int64_t)row * g.Wc;
        for (int x = threadIdx.x; x < g.Wc; x += blockDim.x) o[x] = (float)__ldg(ck + (x >> lb)) * inv;
    }
}

}  // namespace

cudaError_t launch_density(const ImgGeom& g, const int32_t* counts, float* out, cudaStream_t s) {
    const int rows = g.n_img * g.Hc;
    const unsigned grid = (unsigned)(rows < 152 * 8 ? rows : 152 * 8);
    return launch_pdl(density_kernel, dim3(grid > 0 ? grid : 1), dim3(256), 0, s, g, counts, out);
}

cudaError_t setup_ida_fragments() {
    ida_frag_setup_kernel<<<1, 32>>>();
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaDeviceSynchronize();
    return e;
}

int ida_ctas_per_image(const ImgGeom& g) {
    const int NB = kTileCols / g.B;
    return ((g.nbw + NB - 1) / NB) * g.nbh;
}

// The tensor-core step copies x in 16-byte pieces and stores r in pixel
// pairs: x 16-byte, r 8-byte aligned.
static bool ida_tc_usable(const IdaLinArgs& a) {
    return a.g.B == 16 && a.precision != ABCS_FP32 && (reinterpret_cast<uintptr_t>(a.x) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(a.r) & 7) == 0;
}

cudaError_t launch_ida_linear(const IdaLinArgs& a, cudaStream_t s) {
    if (ida_tc_usable(a)) {
        switch (a.precision) {
            case kP16: return launch_lin_tc<kP16>(a, s);
            case kPB16: return launch_lin_tc<kPB16>(a, s);
            case kPB1: return launch_lin_tc<kPB1>(a, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (a.g.B) {
        case 4: return launch_lin_B<4>(a, s);
        case 8: return launch_lin_B<8>(a, s);
        case 16: return launch_lin_B<16>(a, s);
        case 32: return launch_lin_B<32>(a, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_ida_sigma(const IdaLinArgs& a, float* sigma, float* sigma_trace, int iters, int t,
                             cudaStream_t s) {
    const ImgGeom& g = a.g;
    return launch_pdl(ida_sigma_kernel, dim3(g.n_img), dim3(32), 0, s, (const double*)a.partial,
                      ida_ctas_per_image(g), a.offsets, (int64_t)g.n_blocks, sigma, sigma_trace, iters, t,
                      a.status);
}

int damp_chunks(const ImgGeom& g) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const int64_t want = (152 * 8 + g.n_img - 1) / g.n_img, cap = (per_img + 4 * kDampThreads - 1) / (4 * kDampThreads);
    return (int)(want < cap ? (want > 0 ? want : 1) : (cap > 0 ? cap : 1));
}

cudaError_t launch_damp_perturb(const ImgGeom& g, const float* r, const float* probe, float eps_rel,
                                unsigned* amax, float* rp, cudaStream_t s) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const dim3 grid((unsigned)damp_chunks(g), (unsigned)g.n_img);
    cudaError_t e = launch_pdl(damp_clear_kernel, dim3((unsigned)g.n_img), dim3(1), 0, s, amax);
    if (!e) e = launch_pdl(damp_amax_kernel, grid, dim3(kDampThreads), 0, s, r, per_img, amax);
    if (!e)
        e = launch_pdl(damp_perturb_kernel, grid, dim3(kDampThreads), 0, s, r, probe, per_img, (const unsigned*)amax,
                       eps_rel, rp);
    return e;
}

cudaError_t launch_damp_alpha(const ImgGeom& g, const int64_t* offsets, const float* probe, const float* xp,
                              const float* x, const unsigned* amax, float eps_rel, float inv_df, double* partial,
                              float* alpha, float* alpha_trace, int iters, int t, uint32_t* status, cudaStream_t s) {
    const int64_t per_img = (int64_t)g.Hc * g.Wc;
    const int chunks = damp_chunks(g);
    cudaError_t e = launch_pdl(damp_div_kernel, dim3((unsigned)chunks, (unsigned)g.n_img), dim3(kDampThreads), 0, s,
                               probe, xp, x, per_img, partial);
    if (!e)
        e = launch_pdl(damp_alpha_kernel, dim3((unsigned)g.n_img), dim3(32), 0, s, (const double*)partial, chunks,
                       offsets, (int64_t)g.n_blocks, amax, eps_rel, inv_df, alpha, alpha_trace, iters, t, status);
    return e;
}

size_t ida_batch_smem(unsigned used_b_mask) {
    size_t s = kTidctSmem;
    if (used_b_mask & 4) s = s > Tile<4>::smem_bytes(2) ? s : Tile<4>::smem_bytes(2);
    if (used_b_mask & 8) s = s > Tile<8>::smem_bytes(2) ? s : Tile<8>::smem_bytes(2);
    if (used_b_mask & 16) s = s > Tile<16>::smem_bytes(2) ? s : Tile<16>::smem_bytes(2);
    if (used_b_mask & 32) s = s > Tile<32>::smem_bytes(1) ? s : Tile<32>::smem_bytes(1);
    return s;
}

int ida_batch_tile_w() { return kTW; }

template <int TH>
static cudaError_t launch_batch_th(const BatchArgs& a, int ctas_per_sm, size_t smem, cudaStream_t s, int* grid_out) {
    cudaError_t e = cudaFuncSetAttribute(ida_batch_kernel<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int dev, sms, per_sm;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ida_batch_kernel<TH>, 256, smem))) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int use = ctas_per_sm < per_sm ? ctas_per_sm : per_sm;
    int grid = sms * use;
    const int work = a.n_lin > a.n_den ? a.n_lin : a.n_den;
    if (grid > work) grid = work > 0 ? work : 1;
    if (grid_out) *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ida_batch_kernel<TH>, a);
}

// th: denoiser tile height (32 or 64); ctas_per_sm: requested residency
cudaError_t launch_ida_batch(const BatchArgs& a, int th, int ctas_per_sm, size_t smem, cudaStream_t s, int* grid) {
    if (th == 32) return launch_batch_th<32>(a, ctas_per_sm, smem, s, grid);
    return launch_batch_th<64>(a, ctas_per_sm, smem, s, grid);
}

cudaError_t launch_tidct(const float* in, float* out, int n_img, int H, int W, const float* sigma,
                         float lambda, cudaStream_t s) {
    constexpr int TH = 64;
    const size_t smem = kTidctSmem;
    cudaError_t e = cudaFuncSetAttribute(tidct_kernel<TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    dim3 grid((unsigned)((W + kTW - 1) / kTW), (unsigned)((H + TH - 1) / TH), (unsigned)n_img);
    return launch_pdl(tidct_kernel<TH>, grid, dim3(256), smem, s, in, out, H, W, sigma, lambda);
}

}  // namespace abcs
