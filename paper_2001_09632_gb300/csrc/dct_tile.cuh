// Block-row tile helpers shared by the transform kernels (internal).
//
// A CTA of 256 threads owns one block row of one image, 256 pixel columns
// wide: NB = 256 / B blocks side by side.  Two thread mappings are used:
//   row mapping    thread t -> block t / B, pixel row    t % B
//   column mapping thread t -> block t / B, pixel column t % B
// Between the two the block passes through shared memory as Ts[b][r][c]
// with row stride B + 1 (conflict-free in both mappings for B = 4..32).
//
// Include after ABCS_TU_TABLES(...): the transforms read the DCT matrix
// through Dc<B>(k, n) with compile-time indices, i.e. as constant-bank
// operands of the FMAs.
#pragma once

#include "abcs_common.cuh"

namespace abcs {

template <int B>
struct Tile {
    static constexpr int NB = kTileCols / B;   // blocks per CTA
    static constexpr int LD = B + 1;           // padded row stride
    static constexpr int BLK = B * LD;         // floats per block in Ts
    static constexpr int FLOATS = NB * BLK;    // Ts size
    static constexpr int WARPS = 8;
    static constexpr int BPW = NB / WARPS;     // blocks per warp in the packed loops
    static constexpr int PS = NB * B * B + 4;  // floats of one packed staging buffer
    // dynamic shared memory: Ts, `nstage` staging buffers, rank table
    static constexpr size_t smem_bytes(int nstage) {
        return (size_t)(FLOATS + nstage * PS) * 4 + (size_t)B * B * 2;
    }
};

// Carves the dynamic shared memory laid out by Tile<B>::smem_bytes.
template <int B>
struct TileSmem {
    float* Ts;
    float* P[2];
    uint16_t* rk;
    ABCS_D TileSmem(unsigned char* base, int nstage) {
        Ts = reinterpret_cast<float*>(base);
        float* p = Ts + Tile<B>::FLOATS;
        P[0] = p;
        P[1] = nstage > 1 ? p + Tile<B>::PS : p;
        rk = reinterpret_cast<uint16_t*>(p + nstage * Tile<B>::PS);
    }
};

// ---------------------------------------------------------------------------
// 1D orthonormal DCT-II of length B by even/odd folding.
// With D the B-point matrix, N * S = B and x_L the folded input of length N:
//   c[S k] = sum_{n<N} D[S k][n] x_L[n],   and D[S k][N-1-n] = (-1)^k D[S k][n],
// so even k recurse on s[n] = x_L[n] + x_L[N-1-n] (N/2 points, stride 2S)
// and odd k are an (N/2 x N/2) product with d[n] = x_L[n] - x_L[N-1-n].
// 16 points: 86 multiplies + 30 adds instead of 256 multiply-adds.
// ---------------------------------------------------------------------------
template <int B, int S, int N>
ABCS_D void fdct_rec(const float* x, float* c) {
    if constexpr (N == 1) {
        c[0] = Dc<B>(0, 0) * x[0];
    } else {
        constexpr int H = N / 2;
        float s[H], d[H];
#pragma unroll
        for (int n = 0; n < H; ++n) {
            s[n] = x[n] + x[N - 1 - n];
            d[n] = x[n] - x[N - 1 - n];
        }
        fdct_rec<B, 2 * S, H>(s, c);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int n = 0; n < H; ++n) acc = fmaf(Dc<B>(S * (2 * j + 1), n), d[n], acc);
            c[S * (2 * j + 1)] = acc;
        }
    }
}

// Inverse: x_L[n] = sum_{k<N} D[S k][n] c[S k] for n < N; even k give e[n]
// (recursion), odd k give o[n]; x_L[n] = e + o, x_L[N-1-n] = e - o.
template <int B, int S, int N>
ABCS_D void idct_rec(const float* c, float* x) {
    if constexpr (N == 1) {
        x[0] = Dc<B>(0, 0) * c[0];
    } else {
        constexpr int H = N / 2;
        float e[H];
        idct_rec<B, 2 * S, H>(c, e);
#pragma unroll
        for (int n = 0; n < H; ++n) {
            float o = 0.f;
#pragma unroll
            for (int j = 0; j < H; ++j) o = fmaf(Dc<B>(S * (2 * j + 1), n), c[S * (2 * j + 1)], o);
            x[n] = e[n] + o;
            x[N - 1 - n] = e[n] - o;
        }
    }
}

template <int B>
ABCS_D void fdct(const float (&x)[B], float (&c)[B]) { fdct_rec<B, 1, B>(x, c); }
template <int B>
ABCS_D void idct(const float (&c)[B], float (&x)[B]) { idct_rec<B, 1, B>(c, x); }

// ---------------------------------------------------------------------------
// Zigzag tables, one per CTA in smem.
//   load_zz_table:   rank -> padded offset u * (B+1) + v
//   load_rank_table: natural position u * B + v -> rank
// ---------------------------------------------------------------------------
template <int B>
ABCS_D void load_zz_table(uint16_t* zz) {
    for (int i = threadIdx.x; i < B * B; i += blockDim.x) {
        const int p = zz_pos<B>(i);
        zz[i] = (uint16_t)((p / B) * (B + 1) + p % B);
    }
}

template <int B>
ABCS_D void load_rank_table(uint16_t* rk) {
    for (int i = threadIdx.x; i < B * B; i += blockDim.x) rk[zz_pos<B>(i)] = (uint16_t)i;
}

// ---------------------------------------------------------------------------
// Packed ranges staged in shared memory.  A tile's measurements are one
// contiguous range of the packed vector; element e of the range is kept at
// stage[sh + e] with sh = start % 4, so that 16-byte global and shared
// accesses line up (stage itself is 16-byte aligned, 4 floats of slack).
// ---------------------------------------------------------------------------
ABCS_D void stage_in(float* stage, const float* __restrict__ src, int64_t start, int n) {
    const int sh = (int)(start & 3);
    if (reinterpret_cast<uintptr_t>(src) & 15) {     // unaligned base: scalar copy
        for (int e = threadIdx.x; e < n; e += blockDim.x) stage[sh + e] = __ldg(src + start + e);
        return;
    }
    const int head = min(n, (4 - sh) & 3);
    const float* g = src + start;
    for (int e = threadIdx.x; e < head; e += blockDim.x) stage[sh + e] = __ldg(g + e);
    const int nv = (n - head) >> 2;
    const float4* g4 = reinterpret_cast<const float4*>(g + head);
    float4* s4 = reinterpret_cast<float4*>(stage + sh + head);
#pragma unroll 2
    for (int i = threadIdx.x; i < nv; i += blockDim.x) s4[i] = __ldg(g4 + i);
    for (int e = head + 4 * nv + threadIdx.x; e < n; e += blockDim.x) stage[sh + e] = __ldg(g + e);
}

// Same layout as stage_in, copied with cp.async (no registers, no wait):
// the caller commits and waits (cp_async_wait_all) before the barrier that
// publishes the data.
ABCS_D void cp_async4(float* s, const float* g) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(g) : "memory");
}
ABCS_D void cp_async16(float* s, const float* g) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(g) : "memory");
}
ABCS_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
ABCS_D void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
ABCS_D void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory accesses by 32-bit shared addresses (no generic-address
// arithmetic).  The _lt forms take the predicate r < m inside the
// instruction, so a per-coefficient condition costs no branch.
ABCS_D float2 lds_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
ABCS_D float lds_f(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}
// *a if r < m, else 0
ABCS_D float lds_f_lt(uint32_t a, int r, int m) {
    float v;
    // %0 is written before the inputs are read: early clobber
    asm volatile("{\n .reg .pred q;\n setp.lt.s32 q, %2, %3;\n mov.f32 %0, 0f00000000;\n @q ld.shared.f32 %0, [%1];\n}\n"
                 : "=&f"(v)
                 : "r"(a), "r"(r), "r"(m));
    return v;
}
// *a = v if r < m
ABCS_D void sts_f_lt(uint32_t a, float v, int r, int m) {
    asm volatile("{\n .reg .pred q;\n setp.lt.s32 q, %2, %3;\n @q st.shared.f32 [%0], %1;\n}\n" ::"r"(a), "f"(v),
                 "r"(r), "r"(m)
                 : "memory");
}

ABCS_D void stage_in_async(float* stage, const float* __restrict__ src, int64_t start, int n) {
    const int sh = (int)(start & 3);
    const float* g = src + start;
    if (reinterpret_cast<uintptr_t>(src) & 15) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) cp_async4(stage + sh + e, g + e);
        return;
    }
    const int head = min(n, (4 - sh) & 3);
    for (int e = threadIdx.x; e < head; e += blockDim.x) cp_async4(stage + sh + e, g + e);
    const int nv = (n - head) >> 2;
    for (int i = threadIdx.x; i < nv; i += blockDim.x)
        cp_async16(stage + sh + head + 4 * i, g + head + 4 * i);
    for (int e = head + 4 * nv + threadIdx.x; e < n; e += blockDim.x) cp_async4(stage + sh + e, g + e);
}

// The same range of two arrays into two stages in one pass (both sources
// 16-byte aligned, else one array after the other).
ABCS_D void stage_in_async2(float* st1, const float* __restrict__ src1, float* st2, const float* __restrict__ src2,
                            int64_t start, int n) {
    if ((reinterpret_cast<uintptr_t>(src1) | reinterpret_cast<uintptr_t>(src2)) & 15) {
        stage_in_async(st1, src1, start, n);
        stage_in_async(st2, src2, start, n);
        return;
    }
    const int sh = (int)(start & 3);
    const float* g1 = src1 + start;
    const float* g2 = src2 + start;
    const int head = min(n, (4 - sh) & 3);
    for (int e = threadIdx.x; e < head; e += blockDim.x) {
        cp_async4(st1 + sh + e, g1 + e);
        cp_async4(st2 + sh + e, g2 + e);
    }
    const int nv = (n - head) >> 2;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        cp_async16(st1 + sh + head + 4 * i, g1 + head + 4 * i);
        cp_async16(st2 + sh + head + 4 * i, g2 + head + 4 * i);
    }
    for (int e = head + 4 * nv + threadIdx.x; e < n; e += blockDim.x) {
        cp_async4(st1 + sh + e, g1 + e);
        cp_async4(st2 + sh + e, g2 + e);
    }
}

ABCS_D void stage_out(const float* stage, float* __restrict__ dst, int64_t start, int n) {
    const int sh = (int)(start & 3);
    if (reinterpret_cast<uintptr_t>(dst) & 15) {
        for (int e = threadIdx.x; e < n; e += blockDim.x) dst[start + e] = stage[sh + e];
        return;
    }
    const int head = min(n, (4 - sh) & 3);
    float* g = dst + start;
    for (int e = threadIdx.x; e < head; e += blockDim.x) g[e] = stage[sh + e];
    const int nv = (n - head) >> 2;
    float4* g4 = reinterpret_cast<float4*>(g + head);
    const float4* s4 = reinterpret_cast<const float4*>(stage + sh + head);
#pragma unroll 1
    for (int i = threadIdx.x; i < nv; i += blockDim.x) g4[i] = s4[i];
    for (int e = head + 4 * nv + threadIdx.x; e < n; e += blockDim.x) g[e] = stage[sh + e];
}

// ---------------------------------------------------------------------------
// Pixel rows: thread (block b, row n) loads the B pixels of its block row.
// ---------------------------------------------------------------------------
ABCS_D void u8x4_to_f32(uint32_t w, float* f) {
    // byte i -> float via the 2^23 magic number: exact for 0..255
#pragma unroll
    for (int i = 0; i < 4; ++i)
        f[i] = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540 + i)) - 8388608.f;
}

template <int B>
ABCS_D void load_u8_row(const uint8_t* src, bool vec, float (&x)[B]) {
    if (vec) {
        if constexpr (B == 4) {
            u8x4_to_f32(__ldg(reinterpret_cast<const uint32_t*>(src)), x);
        } else if constexpr (B == 8) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(src));
            u8x4_to_f32(v.x, x);
            u8x4_to_f32(v.y, x + 4);
        } else {
#pragma unroll
            for (int q = 0; q < B / 16; ++q) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(src) + q);
                u8x4_to_f32(v.x, x + 16 * q);
                u8x4_to_f32(v.y, x + 16 * q + 4);
                u8x4_to_f32(v.z, x + 16 * q + 8);
                u8x4_to_f32(v.w, x + 16 * q + 12);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = (float)__ldg(src + i);
    }
}

template <int B>
ABCS_D void load_f32_row(const float* src, bool vec, float (&x)[B]) {
    if (vec) {
#pragma unroll
        for (int q = 0; q < B / 4; ++q) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src) + q);
            x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = __ldg(src + i);
    }
}

template <int B>
ABCS_D void store_f32_row(float* dst, bool vec, const float (&x)[B]) {
    if (vec) {
#pragma unroll
        for (int q = 0; q < B / 4; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) dst[i] = x[i];
    }
}

// round half to even, clip to [0, 255]
template <int B>
ABCS_D void store_u8_row(uint8_t* dst, bool vec, const float (&x)[B]) {
    uint8_t b[B];
#pragma unroll
    for (int i = 0; i < B; ++i) b[i] = (uint8_t)fminf(fmaxf(rintf(x[i]), 0.f), 255.f);
    if (vec && B >= 4) {
#pragma unroll
        for (int q = 0; q < B / 4; ++q)
            reinterpret_cast<uint32_t*>(dst)[q] = b[4 * q] | (b[4 * q + 1] << 8) | (b[4 * q + 2] << 16) |
                                                  ((uint32_t)b[4 * q + 3] << 24);
    } else {
#pragma unroll
        for (int i = 0; i < B; ++i) dst[i] = b[i];
    }
}

// ---------------------------------------------------------------------------
// The two halves of the separable 2D transforms on the tile.
// C = D X D^T: rows first (T[n][v] = sum_m X[n][m] D[v][m]), then columns.
// ---------------------------------------------------------------------------
// Row mapping: forward-transform the thread's pixel row into Ts.
template <int B>
ABCS_D void fwd_rows_to_smem(const float (&x)[B], float* Ts) {
    const int b = threadIdx.x / B, n = threadIdx.x % B;
    float c[B];
    fdct<B>(x, c);
    float* row = Ts + b * Tile<B>::BLK + n * Tile<B>::LD;
#pragma unroll
    for (int v = 0; v < B; ++v) row[v] = c[v];
}

// Column mapping, in place: Ts[b][.][v] <- DCT of column v.
template <int B>
ABCS_D void fwd_cols_in_smem(float* Ts) {
    const int b = threadIdx.x / B, v = threadIdx.x % B;
    float* col = Ts + b * Tile<B>::BLK + v;
    float x[B], c[B];
#pragma unroll
    for (int n = 0; n < B; ++n) x[n] = col[n * Tile<B>::LD];
    fdct<B>(x, c);
#pragma unroll
    for (int u = 0; u < B; ++u) col[u * Tile<B>::LD] = c[u];
}

// Column mapping, in place: Ts[b][.][v] <- inverse DCT of column v.
template <int B>
ABCS_D void inv_cols_in_smem(float* Ts) {
    const int b = threadIdx.x / B, v = threadIdx.x % B;
    float* col = Ts + b * Tile<B>::BLK + v;
    float c[B], x[B];
#pragma unroll
    for (int u = 0; u < B; ++u) c[u] = col[u * Tile<B>::LD];
    idct<B>(c, x);
#pragma unroll
    for (int n = 0; n < B; ++n) col[n * Tile<B>::LD] = x[n];
}

// Row mapping: inverse-transform row n of the thread's block from Ts.
template <int B>
ABCS_D void inv_rows_from_smem(const float* Ts, float (&x)[B]) {
    const int b = threadIdx.x / B, n = threadIdx.x % B;
    const float* row = Ts + b * Tile<B>::BLK + n * Tile<B>::LD;
    float c[B];
#pragma unroll
    for (int v = 0; v < B; ++v) c[v] = row[v];
    idct<B>(c, x);
}

// ---------------------------------------------------------------------------
// Called by warp 0 only.  rel[b] = sum_{j<b} c_j for b = 0 .. nblk, with
// c_j = counts[j] clamped to [0, B*B] (a clamp sets ABCS_DEV_BADCOUNT).
// nblk <= 64: lane l owns blocks 2l and 2l+1.
// ---------------------------------------------------------------------------
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

ABCS_D bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace abcs
