// Shared device/host definitions of the ABCS CUDA library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/abcs.h"

#define ABCS_HD __host__ __device__ __forceinline__
#define ABCS_D __device__ __forceinline__

namespace abcs {

// ---------------------------------------------------------------------------
// DCT / zigzag tables.  Every translation unit that runs transforms keeps its
// own copy in __constant__ memory; abcs_create() uploads them (per device).
// Indices are compile-time constants inside the unrolled transforms, so the
// coefficients become constant-bank operands of the FMAs.
// ---------------------------------------------------------------------------
struct HostTables {
    float Df4[16], Df8[64], Df16[256], Df32[1024];          // D[k][n], orthonormal DCT-II
    double Dd4[16], Dd8[64], Dd16[256], Dd32[1024];
    uint16_t zzpos4[16], zzpos8[64], zzpos16[256], zzpos32[1024];   // rank -> u*B + v
};
const HostTables& host_tables();   // computed once on the host in double

#define ABCS_TU_TABLES(NAME)                                                        \
    static __constant__ float c_Df4[16], c_Df8[64], c_Df16[256], c_Df32[1024];       \
    static __constant__ double c_Dd4[16], c_Dd8[64], c_Dd16[256], c_Dd32[1024];      \
    static __constant__ uint16_t c_zz4[16], c_zz8[64], c_zz16[256], c_zz32[1024];    \
    cudaError_t upload_tables_##NAME() {                                             \
        const HostTables& t = host_tables();                                         \
        cudaError_t e = cudaSuccess;                                                 \
        if (!e) e = cudaMemcpyToSymbol(c_Df4, t.Df4, sizeof t.Df4);                  \
        if (!e) e = cudaMemcpyToSymbol(c_Df8, t.Df8, sizeof t.Df8);                  \
        if (!e) e = cudaMemcpyToSymbol(c_Df16, t.Df16, sizeof t.Df16);               \
        if (!e) e = cudaMemcpyToSymbol(c_Df32, t.Df32, sizeof t.Df32);               \
        if (!e) e = cudaMemcpyToSymbol(c_Dd4, t.Dd4, sizeof t.Dd4);                  \
        if (!e) e = cudaMemcpyToSymbol(c_Dd8, t.Dd8, sizeof t.Dd8);                  \
        if (!e) e = cudaMemcpyToSymbol(c_Dd16, t.Dd16, sizeof t.Dd16);               \
        if (!e) e = cudaMemcpyToSymbol(c_Dd32, t.Dd32, sizeof t.Dd32);               \
        if (!e) e = cudaMemcpyToSymbol(c_zz4, t.zzpos4, sizeof t.zzpos4);            \
        if (!e) e = cudaMemcpyToSymbol(c_zz8, t.zzpos8, sizeof t.zzpos8);            \
        if (!e) e = cudaMemcpyToSymbol(c_zz16, t.zzpos16, sizeof t.zzpos16);         \
        if (!e) e = cudaMemcpyToSymbol(c_zz32, t.zzpos32, sizeof t.zzpos32);         \
        return e;                                                                    \
    }                                                                                \
    template <int B> ABCS_D float Dc(int k, int n) {                                 \
        if constexpr (B == 4) return c_Df4[k * 4 + n];                               \
        else if constexpr (B == 8) return c_Df8[k * 8 + n];                          \
        else if constexpr (B == 16) return c_Df16[k * 16 + n];                       \
        else return c_Df32[k * 32 + n];                                              \
    }                                                                                \
    template <int B> ABCS_D double Dd(int k, int n) {                                \
        if constexpr (B == 4) return c_Dd4[k * 4 + n];                               \
        else if constexpr (B == 8) return c_Dd8[k * 8 + n];                          \
        else if constexpr (B == 16) return c_Dd16[k * 16 + n];                       \
        else return c_Dd32[k * 32 + n];                                              \
    }                                                                                \
    template <int B> ABCS_D int zz_pos(int rank) {                                   \
        if constexpr (B == 4) return c_zz4[rank];                                    \
        else if constexpr (B == 8) return c_zz8[rank];                               \
        else if constexpr (B == 16) return c_zz16[rank];                             \
        else return c_zz32[rank];                                                    \
    }

cudaError_t upload_tables_pilot();
cudaError_t upload_tables_dct();
cudaError_t upload_tables_ida();
cudaError_t upload_tables_tc();
cudaError_t upload_tables_su();
cudaError_t setup_tc_fragments();   // after upload_tables_tc(), per device
cudaError_t setup_sense_umma();     // after upload_tables_su(), per device

// zigzag rank of (u, v) in a B x B block, JPEG orientation: diagonal s = u+v;
// odd s runs with u increasing, even s with u decreasing.
ABCS_HD int zz_rank(int u, int v, int B) {
    const int s = u + v;
    if (s < B) {
        const int base = s * (s + 1) / 2;
        return base + ((s & 1) ? u : (s - u));
    }
    const int rem = 2 * B - 1 - s;                 // entries on diagonal s
    const int base = B * B - rem * (rem + 1) / 2;
    return base + ((s & 1) ? (u - (s - B + 1)) : (B - 1 - u));
}

// ---------------------------------------------------------------------------
// Launch geometry shared by the block-transform kernels: a CTA covers one
// block row of one image, 256 pixel columns wide (256 / B blocks), one
// thread per pixel column.
// ---------------------------------------------------------------------------
constexpr int kTileCols = 256;

struct ImgGeom {
    int n_img;
    int H, W;          // original image size (pixels)
    int B;
    int nbh, nbw;      // block grid after cropping
    int Hc, Wc;        // cropped size
    int64_t n_blocks;  // per image
    int64_t pitch;     // bytes between rows (uint8 inputs)
    int64_t img_stride;// bytes between images (uint8 inputs)
};

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while its predecessor in the stream drains; it must call griddep_wait()
// before touching any global memory the predecessor may write (all inputs).
ABCS_D void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// Lets the next kernel of the stream (launched with launch_pdl) start its
// CTAs before this grid ends.  Called only after this kernel's own
// griddep_wait(), so everything before it in the stream is complete by then.
ABCS_D void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Device status bits are OR-ed into one word owned by the handle.
ABCS_D void set_status(uint32_t* st, uint32_t bits) { atomicOr(st, bits); }

template <typename T>
ABCS_D T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a CTA of blockDim.x threads (multiple of 32, <= 1024).  `sh` needs
// 32 elements.  The result is valid in every thread.  Fixed order.
template <typename T>
ABCS_D T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T t = (lane < nw) ? sh[lane] : T(0);
    t = warp_sum(t);
    return t;
}

}  // namespace abcs

// Launchers (host side, one per translation unit).
namespace abcs {
struct SenseArgs {
    ImgGeom g;
    const uint8_t* img;
    int variant, precision;
    int L, X0, nS, m1, m_zz, T, cap;
    int64_t R;
    int32_t* counts;
    int64_t* offsets;
    float* coeffs;
    int64_t capacity;
    int32_t* w;          // pilot per block (BBV_i or n_i)
    unsigned long long* wpart;  // per image, per pilot CTA: partial sums of w
    int pilot_cpi;       // pilot CTAs per image (partials per image)
    int64_t* img_total;  // per image sum of counts
    int64_t* img_base;   // exclusive prefix of img_total, n_img + 1 entries
    unsigned* done;      // allocation CTAs finished (reset by the last one)
    unsigned* img_done;  // per image: pilot CTAs finished (fused allocation; reset after use), or NULL
    uint32_t* status;
    int pilot_bases;     // 1: the allocation writes img_base; 0: the sensing kernel derives the
                         // image bases from img_total itself (tensor-core sensing kernels)
};
// Uneven batch (abcs_sense_batch): one entry per image, in batch order.
struct SenseBatchImg {
    ImgGeom g;           // the image alone (n_img = 1)
    int64_t img_off;     // byte offset of its first pixel
    int64_t blk0;        // its first block in counts / offsets / pilot
    int variant, L, X0, nS, m1, m_zz, T, cap;
    int64_t R;
    int mode;            // pilot: 1 BBV, 2 DD; allocation only: 0 (ZZ), 3 (BBV with n_S = 0)
    int item0, cpi;      // its first pilot work item and their number
    int tile0;           // its first sensing tile
};

struct SenseBatchArgs {
    const SenseBatchImg* imgs;
    int n_img;
    const uint8_t* img;
    int32_t* counts;
    int64_t* offsets;
    float* coeffs;
    int64_t capacity;
    int32_t* w;                 // pilot values, one per block
    unsigned long long* wpart;  // one per pilot work item
    int64_t* img_total;
    int64_t* img_base;
    unsigned* done;
    unsigned* img_done;
    uint32_t* status;
};

// The arguments of image k of a batch as a one-image SenseArgs: its blocks,
// counts, offsets and pilot values start at the image's first block.
ABCS_D SenseArgs batch_image_args(const SenseBatchArgs& b, const SenseBatchImg& e, int k) {
    SenseArgs a{};
    a.g = e.g;
    a.img = b.img + e.img_off;
    a.variant = e.variant;
    a.precision = ABCS_FP32;
    a.L = e.L; a.X0 = e.X0; a.nS = e.nS; a.m1 = e.m1; a.m_zz = e.m_zz; a.T = e.T; a.cap = e.cap;
    a.R = e.R;
    a.counts = b.counts + e.blk0;
    a.offsets = b.offsets + e.blk0;
    a.coeffs = b.coeffs;
    a.capacity = b.capacity;
    a.w = b.w + e.blk0;
    a.wpart = b.wpart + e.item0;
    a.pilot_cpi = e.cpi;
    a.img_total = b.img_total + k;
    a.img_base = b.img_base + k;
    a.done = b.done;
    a.img_done = b.img_done + k;
    a.status = b.status;
    a.pilot_bases = 0;
    return a;
}

cudaError_t launch_pilot_batch(const SenseBatchArgs& b, int n_items, cudaStream_t s);
cudaError_t launch_sense_batch(const SenseBatchArgs& b, int n_tiles, cudaStream_t s);
int pilot_ctas_per_image(const SenseArgs& a);
cudaError_t launch_bbv_pilot(const SenseArgs& a, cudaStream_t s);
cudaError_t launch_dd_pilot(const SenseArgs& a, cudaStream_t s);
cudaError_t launch_allocate(const SenseArgs& a, int mode, cudaStream_t s);
// pilot + allocation in one launch (needs a.img_done, zero on entry)
cudaError_t launch_bbv_alloc(const SenseArgs& a, cudaStream_t s);
cudaError_t launch_dd_alloc(const SenseArgs& a, cudaStream_t s);
// DD pilot + allocation on the tensor cores (k_tc.cu; B = 16, 4-byte aligned pixel rows)
bool dd_tc_usable(const SenseArgs& a);
cudaError_t launch_dd_tc_alloc(const SenseArgs& a, cudaStream_t s);
cudaError_t launch_sense_pack(const SenseArgs& a, cudaStream_t s);

struct ReconArgs {
    ImgGeom g;
    int precision;
    const int32_t* counts;
    const int64_t* offsets;
    const float* coeffs;
    float* out;
    uint8_t* out_u8;
    uint32_t* status;
};
cudaError_t launch_reconstruct(const ReconArgs& a, cudaStream_t s);
// tensor-core paths (B = 16; a.precision selects FP16x2 / BF16x2 / BF16)
cudaError_t launch_sense_tc(const SenseArgs& a, cudaStream_t s);
// whether the mma.sync sensing kernel can derive the image bases itself
// (its CTAs' block ranges span at most 64 images)
bool sense_tc_bases_in_kernel(const SenseArgs& a);
// tcgen05 sensing (k_sense_umma.cu): B = 16, 16-byte aligned images and rows
bool sense_umma_usable(const SenseArgs& a);
cudaError_t launch_sense_umma(const SenseArgs& a, cudaStream_t s);
cudaError_t launch_recon_tc(const ReconArgs& a, cudaStream_t s);

struct IdaLinArgs {
    ImgGeom g;
    const int32_t* counts;
    const int64_t* offsets;
    const float* y;
    const float* x;        // NULL: x = 0
    const float* z_prev;   // NULL: z_prev = 0
    float* z;
    float* r;
    double* partial;       // one per CTA
    float inv_df;          // Onsager coefficient of IDA (Eq. 28) ...
    const float* alpha;    // ... or per image (D-AMP / DAMP-D, Eqs. 24, 27), if not NULL
    uint32_t* status;
    int precision;         // abcs_precision: tensor-core transforms for B = 16 (aligned x, r)
};
cudaError_t launch_ida_linear(const IdaLinArgs& a, cudaStream_t s);
cudaError_t setup_ida_fragments();   // after upload_tables_ida(), per device
// D-AMP / DAMP-D Onsager coefficient (k_ida.cu): per image
//   alpha[k] = inv_df * div_k / M_k,  div_k = b^T (xp - x) / eps_k,  eps_k = eps_rel max|r|
// amax: n_img words (cleared here); partial: n_img x chunks doubles
cudaError_t launch_damp_perturb(const ImgGeom& g, const float* r, const float* probe, float eps_rel,
                                unsigned* amax, float* rp, cudaStream_t s);
cudaError_t launch_damp_alpha(const ImgGeom& g, const int64_t* offsets, const float* probe, const float* xp,
                              const float* x, const unsigned* amax, float eps_rel, float inv_df, double* partial,
                              float* alpha, float* alpha_trace, int iters, int t, uint32_t* status, cudaStream_t s);
int damp_chunks(const ImgGeom& g);
// sigma^t per image from the partials of the linear step just launched with `a`
cudaError_t launch_ida_sigma(const IdaLinArgs& a, float* sigma, float* sigma_trace, int iters, int t,
                             cudaStream_t s);
int ida_ctas_per_image(const ImgGeom& g);
cudaError_t launch_tidct(const float* in, float* out, int n_img, int H, int W, const float* sigma,
                         float lambda, cudaStream_t s);

// Uneven IDA batch (k_ida.cu): per-image geometry and the persistent kernel's arguments.
struct BatchImg {
    int Hc, Wc, B, nbw, nbh;
    int lin0, den0;            // first linear / denoiser tile of the image
    int64_t blk0;              // first block in counts / offsets
    int64_t pix0;              // first pixel in x / r
    int64_t coeff_base;        // added to offsets
};

struct BatchArgs {
    const BatchImg* imgs;
    int n_img, n_lin, n_den, iters, denoiser;
    const int32_t* counts;
    const int64_t* offsets;
    const float* y;
    float* x;
    float* r0;
    float* r1;
    float* z0;
    float* z1;
    double* partial;           // one per linear tile
    float* sigma;              // one per image
    float* trace;              // [n_img][iters] or NULL
    float inv_df, lambda;
    uint32_t* status;
    unsigned* bar;             // arrival count, generation, abort flag
    long long timeout;
    int skip_cta;              // failure-detection test: this CTA skips its first arrival (-1: none)
};

size_t ida_batch_smem(unsigned used_b_mask);
int ida_batch_tile_w();
cudaError_t launch_ida_batch(const BatchArgs& a, int th, int ctas_per_sm, size_t smem, cudaStream_t s, int* grid);

// learned denoiser (k_cnn.cu)
int cnn_param_count();
size_t cnn_packed_bytes();
cudaError_t cnn_pack(const float* params, void* packed, cudaStream_t s);
// tau: the iteration input per image, or NULL for tau0 in every image
cudaError_t cnn_forward(const void* packed, const float* r, const float* sigma, const float* dens, const float* tau,
                        float tau0, int n, int H, int W, void* act_buf, int keep_all, int mode, float* out,
                        uint32_t* status, cudaStream_t s);
cudaError_t cnn_grad(const void* packed, const float* r, const float* clean, const float* sigma, const float* dens,
                     const float* tau, int n, int H, int W, void* ws, float* grad, float* loss, uint32_t* status,
                     cudaStream_t s);
// the learned denoiser's iteration input in IDA iteration t
inline float cnn_iter_input(int t) { return (float)(t < 8 ? t : 8) / 8.f; }
// PSNR and SSIM per image (k_quality.cu): x [n][H][W] float, ref uint8 with
// row pitch and image stride; psnr, ssim [n] double; H, W >= 11
cudaError_t setup_quality_tables();
size_t quality_ws_bytes(int n_img, int H, int W);
cudaError_t launch_psnr_ssim(const float* x, const uint8_t* ref, int n_img, int H, int W, int64_t pitch,
                             int64_t stride, double* psnr, double* ssim, void* ws, cudaStream_t s);
// per-pixel measured fraction m_i / B^2 of the pixel's block (k_ida.cu)
cudaError_t launch_density(const ImgGeom& g, const int32_t* counts, float* out, cudaStream_t s);
// BM3D hard-thresholding step (k_bm3d.cu): in, out [n_img][H][W]; num, den
// workspace of the same size; tables uploaded once per device
cudaError_t setup_bm3d_tables();
cudaError_t launch_bm3d(const float* in, float* out, int n_img, int H, int W, const float* sigma, float lambda,
                        float* num, float* den, cudaStream_t s);
// THI selection (k_thi.cu): coeffs n_img x nB x bb (zigzag rank order);
// workspace prefix/rem (n_img), hist (n_img x 256), gt/eq (n_img x nB)
cudaError_t launch_thi(const float* coeffs, int n_img, int nB, int bb, int64_t M, const int32_t* adaptive,
                       int32_t* counts, double* rho, float* masked, uint32_t* prefix, int64_t* rem, uint32_t* hist,
                       int32_t* gt, int32_t* eq, uint32_t* status, cudaStream_t s);
size_t cnn_grad_ws_bytes(int n, int H, int W);
cudaError_t cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr, cudaStream_t s);
}  // namespace abcs
