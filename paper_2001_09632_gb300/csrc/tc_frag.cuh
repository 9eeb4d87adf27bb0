// Operand helpers of the per-block tensor-core transforms (B = 16) on
// mma.sync.m16n8k16 with FP32 accumulation: packing and hi + lo splitting
// of FP32 values into FP16 or BF16 pairs, the MMA wrappers and the fragment
// coordinates.  Include after the translation unit's DCT tables (Dd<16>).
//   TC_FP16X2  v = hi + lo in FP16; products hi*hi + lo*hi + hi*lo
//   TC_BF16X2  the same split in BF16
//   TC_BF16    single BF16 product hi*hi
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "abcs_common.cuh"

namespace abcs {

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

// index of a tensor-core precision in per-precision tables
template <int P>
__host__ __device__ constexpr int pidx() { return P == kP16 ? 0 : (P == kPB16 ? 1 : 2); }

}  // namespace abcs
