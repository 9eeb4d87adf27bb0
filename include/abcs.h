/*
 * abcs.h -- C ABI of the GB300 (sm_103a) adaptive block compressive sensing
 * (ABCS) library, libabcs.so.
 *
 * The operations follow Zammit & Wassell, "Adaptive Block Compressive
 * Sensing: towards a real-time and low-complexity implementation"
 * (arXiv 2001.09632):
 *   abcs_plan ............ derived scalars, Eqs. 16-18, 20-21, Alg. 2 step 2, Table 1
 *   abcs_sense ........... Alg. 1 (AL-DCT-BBV) / Alg. 2 (AL-DCT-DD) / L-DCT-ZZ (Sec. IV):
 *                          pilot estimate (Eq. 19 or Sec. V-B), allocation (Eqs. 22-23),
 *                          zigzag-ordered 2D-DCT measurements (Eq. 26 rows)
 *   abcs_sense_batch ..... the same over images of different sizes, block sizes,
 *                          variants and subrates, two launches per batch
 *   abcs_reconstruct ..... the real-time decoder output I_o of Fig. 1: block inverse
 *                          2D-DCT of the zero-filled measurements (Sec. VII-D)
 *   abcs_ida ............. IDA, Eqs. 13, 15, 25 with alpha = 1/D_F (Eq. 28)
 *   abcs_denoise_tidct ... the plain denoiser D_sigma used inside IDA (Sec. VI-4 names
 *                          BM3D / DnCNN; this library's plain stand-in is
 *                          shift-averaged 8x8 DCT hard thresholding)
 *   abcs_cnn_* ........... the learned residual CNN denoiser (DnCNN-style, Sec. VI-4)
 *   abcs_psnr_ssim ....... the quality measures of the paper's tables (PSNR, SSIM of ref. [18])
 *
 * Conventions shared by every entry point:
 *   - Pointers marked [device] are CUDA device pointers (or managed memory)
 *     allocated and owned by the caller; the library never frees them and
 *     keeps no reference after the call returns.  [host] pointers are read or
 *     written before the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work of a call is enqueued on that stream in
 *     order; the call does not synchronise unless stated.
 *   - Images are greyscale uint8, row-major; image k of a batch starts at
 *     img + k * img_stride and row r at + r * pitch (both in bytes).  Only the
 *     top-left floor(H/B)*B x floor(W/B)*B crop is sensed (Alg. 1/2 step 1).
 *   - Blocks are numbered row-major inside an image; image k's blocks follow
 *     image k-1's.  counts[k*n_B + i] = m_i of block i of image k;
 *     offsets has n_img*n_B + 1 entries, offsets[j] = sum of counts before
 *     block j (global over the batch), offsets[last] = total measurements.
 *     coeffs[offsets[j] + t], t < counts[j], is block j's zigzag-rank-t
 *     orthonormal DCT coefficient (JPEG zigzag orientation).
 *   - Float images written by the library are dense float32
 *     [n_img][floor(H/B)*B][floor(W/B)*B].
 *   - Return values are abcs_status; no exception crosses the ABI.  A
 *     non-OK return leaves a message for abcs_last_error() (thread-local).
 *     Argument errors are detected before any device work is enqueued.
 *     Conditions only the device can see (capacity overrun, non-finite
 *     IDA residual, undecidable DD tie, spin timeout) set bits in the
 *     handle's device status word, read by abcs_sync_status().
 */
#ifndef ABCS_H
#define ABCS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ABCS_API_VERSION 1

typedef enum abcs_status {
    ABCS_OK = 0,
    ABCS_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or geometry */
    ABCS_ERR_UNSUPPORTED = 2,   /* valid request the method does not define (e.g. BBV with L = 1) */
    ABCS_ERR_CAPACITY = 3,      /* an output buffer is smaller than the bound the call needs */
    ABCS_ERR_OOM = 4,           /* library workspace allocation failed */
    ABCS_ERR_CUDA = 5,          /* a CUDA runtime call failed (message has the CUDA error) */
    ABCS_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    ABCS_ERR_NONFINITE = 7,     /* IDA met a non-finite residual norm */
    ABCS_ERR_DEVICE = 8         /* abcs_sync_status: device status bits were set */
} abcs_status;

/* Bits of the device status word (abcs_sync_status). */
#define ABCS_DEV_CAPACITY  0x1u  /* a kernel skipped writes beyond coeff_capacity */
#define ABCS_DEV_AMBIGUOUS 0x2u  /* a DD pilot coefficient within 1e-9 of T that is not exactly decidable */
#define ABCS_DEV_NONFINITE 0x4u  /* IDA: ||z||^2 not finite for some image */
#define ABCS_DEV_TIMEOUT   0x8u  /* a bounded spin-wait expired */
#define ABCS_DEV_BADCOUNT  0x10u /* a count outside [0, B*B] was clamped */

typedef enum abcs_variant {
    ABCS_ZZ = 0,    /* non-adaptive L-DCT-ZZ: floor(B^2 subrate) coefficients per block (Eq. 26) */
    ABCS_BBV = 1,   /* AL-DCT-BBV, Alg. 1 */
    ABCS_DD = 2     /* AL-DCT-DD, Alg. 2 */
} abcs_variant;

typedef enum abcs_precision {
    ABCS_FP32 = 0,        /* FP32 CUDA-core transforms */
    ABCS_TC_FP16X2 = 1,   /* tensor-core FP16 hi+lo split products, FP32 accumulate (B = 16) */
    ABCS_TC_BF16X2 = 2,   /* tensor-core BF16 hi+lo split products, FP32 accumulate (B = 16) */
    ABCS_TC_BF16 = 3      /* tensor-core single BF16 product, FP32 accumulate (B = 16) */
} abcs_precision;

typedef enum abcs_denoiser {
    ABCS_DEN_NONE = 0,    /* identity: x^{t+1} = x^t + A^T z^t (used to check the linear part) */
    ABCS_DEN_TIDCT = 1,   /* plain: shift-averaged 8x8 DCT hard thresholding at lambda * sigma */
    ABCS_DEN_CNN = 2,     /* learned: residual CNN, weights from abcs_cnn_* */
    ABCS_DEN_BM3D = 3     /* plain: BM3D's hard-thresholding step (abcs_bm3d_denoise); lambda = lambda_3D */
} abcs_denoiser;

typedef struct abcs_handle abcs_handle;

/* Derived scalars of one image (abcs_plan). */
typedef struct abcs_plan_info {
    int32_t H, W, B, variant;
    int32_t nbh, nbw;          /* blocks per column / row after cropping (Eq. 20) */
    int64_t n_blocks;          /* n_B = nbh * nbw */
    int64_t N;                 /* cropped pixels n_B * B^2 */
    int64_t M;                 /* floor(subrate * N) measurement budget */
    double CF;                 /* compression factor 1 / subrate */
    int32_t L, X0, nS;         /* Eqs. 16-18 (BBV sampling stride, offset, samples per side) */
    int32_t m1;                /* phase-1 measurements per block: BBV 2 n_S, DD floor(B^2/(2 C_F)), ZZ 0 */
    int32_t m_zz;              /* floor(B^2 subrate): L-DCT-ZZ count */
    int32_t T;                 /* DD threshold (Table 1); 0 otherwise */
    int32_t cap;               /* cap of m_i^2: B^2 - m1 */
    int64_t M_bbv;             /* pixel differences measured by BBV (Eq. 21 as measured) */
    int64_t R;                 /* phase-2 budget: BBV M - M_bbv, DD n_B m1 */
    int64_t max_coeffs;        /* upper bound of sum m_i for this image (== M) */
} abcs_plan_info;

/* Create a handle bound to the current CUDA device.  It owns a device
 * status word and a workspace grown on demand (cudaMalloc; growing waits
 * for the device).  Uploads the DCT and zigzag tables to this device.
 * Failure-detection test hooks, read from the environment at each call
 * (host-side; nothing faults or hangs):
 *   ABCS_FAULT_WS_LIMIT=n     a workspace larger than n bytes fails with
 *                             ABCS_ERR_OOM, as a failed allocation would;
 *   ABCS_FAULT_SKIP_ARRIVE=k  in abcs_ida_batch, CTA k waits at its first
 *                             grid barrier without arriving, so the bounded
 *                             waits expire (ABCS_DEV_TIMEOUT). */
abcs_status abcs_create(abcs_handle** out);

/* Free the handle's device memory.  Waits for the device first.  NULL is a no-op. */
void abcs_destroy(abcs_handle* h);

/* Message of the last failed call on this thread ("" if none). */
const char* abcs_last_error(void);

/* Host only, no device work.  Computes the scalars of one H x W image for
 * block size B (4, 8, 16 or 32), subrate in (0, 1] and a variant.
 * INVALID_ARG: H < B, W < B, bad B or subrate, NULL out.
 * UNSUPPORTED: BBV with L = floor(1/subrate) = 1 (Eq. 17 puts the first
 * sample at column 0, outside the block). */
abcs_status abcs_plan(int H, int W, int B, double subrate, int variant, abcs_plan_info* out);

/* Sense a batch of n_img equally sized images (Alg. 1 / Alg. 2).
 *   img      [device] uint8, see conventions (pitch, img_stride in bytes)
 *   counts   [device] int32  [n_img * n_B]      out: m_i per block
 *   offsets  [device] int64  [n_img * n_B + 1]  out: exclusive prefix of counts
 *   coeffs   [device] float  [coeff_capacity]   out: packed measurements
 *   pilot    [device] int32  [n_img * n_B] or NULL; out: BBV_i (BBV) or n_i (DD)
 * coeff_capacity must be >= n_img * plan.M (the sum of m_i never exceeds M
 * per image), else ABCS_ERR_CAPACITY before any work.  Counts are exact
 * integers; the DD decisions |c| > T are taken on the exact coefficient.
 * precision selects how the measured coefficients are computed; pilot
 * decisions do not depend on it.  Tensor-core precisions (B = 16) run the
 * per-block mma.sync transform; with the environment variable
 * ABCS_SENSE_TC=umma (read at each call) and 16-byte aligned img, pitch and
 * img_stride they run the tcgen05 kernel instead, which computes each
 * 64-block tile as one GEMM against the zigzag-ordered DCT basis (the same
 * results within the precision's bound; slower on the measured workloads). */
abcs_status abcs_sense(abcs_handle* h, const uint8_t* img, int n_img, int H, int W,
                       int64_t pitch, int64_t img_stride, int B, double subrate,
                       int variant, int precision, int32_t* counts, int64_t* offsets,
                       float* coeffs, int64_t coeff_capacity, int32_t* pilot, void* stream);

/* One image of an uneven sensing batch (abcs_sense_batch). */
typedef struct abcs_sense_desc {
    int32_t H, W, B;         /* image size in pixels, block size (4, 8, 16 or 32) */
    int32_t variant;         /* abcs_variant */
    double subrate;          /* (0, 1] */
    int64_t img_offset;      /* byte offset of the image's first pixel from `img` */
    int64_t pitch;           /* bytes between the image's rows (>= W) */
} abcs_sense_desc;

/* Sense a batch of images of different sizes, block sizes, variants and
 * subrates (Alg. 1 / Alg. 2 per image, as abcs_sense computes them), in two
 * launches for the whole batch: one for every image's pilot estimate and
 * allocation (Eq. 19 or Sec. V-B; Eqs. 22-23), one for every image's
 * measurements (Eq. 26 rows).
 *   img      [device] uint8; image k at img + desc[k].img_offset, rows desc[k].pitch apart
 *   desc     [host] n_img descriptors
 *   counts   [device] int32  [total blocks]      out: m_i per block
 *   offsets  [device] int64  [total blocks + 1]  out: exclusive prefix of counts over the batch
 *   coeffs   [device] float  [coeff_capacity]    out: packed measurements
 *   pilot    [device] int32  [total blocks] or NULL; out: BBV_i / n_i (0 for L-DCT-ZZ)
 * Image k's blocks follow image k-1's (raster order within an image), so
 * image k's first block is the sum of n_B over the images before it and its
 * measurements start at offsets[that block]; total blocks = the sum of the
 * images' n_B.  The layout is the one abcs_ida_batch reads (block_offset =
 * the image's first block, coeff_base = 0).  precision: ABCS_FP32 only (a
 * tensor-core precision returns ABCS_ERR_UNSUPPORTED).  coeff_capacity must
 * be >= the sum of the images' plan.M, else ABCS_ERR_CAPACITY before any
 * work.  A descriptor abcs_plan rejects fails the call with that status. */
abcs_status abcs_sense_batch(abcs_handle* h, const uint8_t* img, const abcs_sense_desc* desc, int n_img,
                             int precision, int32_t* counts, int64_t* offsets, float* coeffs,
                             int64_t coeff_capacity, int32_t* pilot, void* stream);

/* Block inverse 2D-DCT of the zero-filled measurements (A^T y, Fig. 1 I_o).
 *   counts, offsets, coeffs [device] as written by abcs_sense
 *   out     [device] float [n_img][Hc][Wc] (Hc = floor(H/B) B, Wc = floor(W/B) B), or NULL
 *   out_u8  [device] uint8 [n_img][Hc][Wc] rounded half-to-even and clipped to [0,255], or NULL
 * At least one of out / out_u8 must be non-NULL.  Counts outside [0, B^2]
 * are clamped and flagged (ABCS_DEV_BADCOUNT).
 * Tensor-core precisions (B = 16) run the per-block mma.sync transform; with
 * the environment variable ABCS_RECON_TC=umma (read at each call) they run
 * the tcgen05 kernel instead, which computes each 128-block tile as one GEMM
 * against the DCT basis images held in tensor memory (same results within
 * the precision's bound; slower on the measured workloads). */
abcs_status abcs_reconstruct(abcs_handle* h, const int32_t* counts, const int64_t* offsets,
                             const float* coeffs, int n_img, int H, int W, int B, int precision,
                             float* out, uint8_t* out_u8, void* stream);

/* IDA (Sec. VI): x^0 = 0, z^{-1} = 0; for t < iters:
 *   z^t = y - A x^t + z^{t-1} / damping,   sigma^t = sqrt(||z^t||^2 / m_img),
 *   x^{t+1} = D_{sigma^t}(x^t + A^T z^t).
 *   counts, offsets, y [device] as written by abcs_sense (m_img = the image's
 *                      number of measurements)
 *   denoiser           abcs_denoiser; lambda is the TI-DCT threshold factor (2.3 here) or
 *                      BM3D's lambda_3D (2.7)
 *   cnn_weights        [device] packed weights of abcs_cnn_* (ABCS_DEN_CNN) or NULL
 *   x_out              [device] float [n_img][Hc][Wc], out: x^iters
 *   sigma_trace        [device] float [n_img][iters] or NULL, out: sigma^t
 * A non-finite sigma sets ABCS_DEV_NONFINITE; that image's later iterates
 * are not meaningful. */
abcs_status abcs_ida(abcs_handle* h, const int32_t* counts, const int64_t* offsets,
                     const float* y, int n_img, int H, int W, int B, int iters, double damping,
                     int denoiser, double lambda, const void* cnn_weights,
                     float* x_out, float* sigma_trace, void* stream);

/* The paper's two quality measures (PSNR and SSIM, Tables 3, 6, 7) of
 * reconstructions against the clean images, per image, with x clipped to
 * [0, 255]:
 *   PSNR = 10 log10(255^2 / MSE)  (+infinity when MSE = 0),
 *   SSIM = mean over the valid (unpadded) region of Wang et al.'s map with
 *          an 11 x 11 Gaussian window (sigma 1.5), K1 = 0.01, K2 = 0.03,
 *          L = 255.
 *   x          [device] float [n_img][H][W]
 *   ref        [device] uint8: image k, row y at ref + k ref_stride + y ref_pitch
 *   psnr, ssim [device] double [n_img], out
 * H, W >= 11, ref_pitch >= W, ref_stride >= ref_pitch H (n_img > 1);
 * otherwise ABCS_ERR_INVALID_ARG.  Uses the handle's workspace. */
abcs_status abcs_psnr_ssim(abcs_handle* h, const float* x, const uint8_t* ref, int n_img, int H, int W,
                           int64_t ref_pitch, int64_t ref_stride, double* psnr, double* ssim, void* stream);

/* Transform precision of the IDA linear step (Eqs. 25, 28: A x and A^T z)
 * in abcs_ida, abcs_damp and abcs_ida_capture on this handle.  ABCS_FP32
 * (the default) runs FP32 CUDA-core butterflies for every block size.  A
 * tensor-core precision runs, for B = 16, the per-block mma.sync transform
 * (r = x + D^T Z D of the masked residual Z, so x's unmeasured components
 * pass unchanged; ||z||^2 is summed in FP32 per lane over at most 16 terms,
 * then in FP64); other block sizes, and x or x_out not 8-byte aligned, keep
 * FP32.  abcs_ida_batch always runs FP32.
 * Returns ABCS_ERR_INVALID_ARG for a NULL handle or an unknown precision. */
abcs_status abcs_set_ida_precision(abcs_handle* h, int precision);

/* D-AMP (Eq. 24) and its damped form DAMP-D (Eq. 27): IDA with the Onsager
 * coefficient taken from the denoiser's divergence instead of 1 / damping:
 *   z^t = y - A x^t + alpha^t z^{t-1},
 *   alpha^t = div[D_{sigma^{t-1}}(r^{t-1})] / (m_img damping),  alpha^0 = 0,
 * damping = 1 gives D-AMP.  The divergence is the Monte-Carlo estimate
 *   div ~ b^T (D(r + eps b) - D(r)) / eps,  eps = max|r| / 1000 per image,
 * with the caller's probe b, so every iteration but the last runs the
 * denoiser twice.  (The paper's (1/delta) div / m is read as AMP's
 * (1/delta) <eta'> = div / m_img.)
 *   probe       [device] float [n_img][Hc][Wc], e.g. +-1 entries
 *   alpha_trace [device] float [n_img][iters] or NULL, out: alpha^t
 * Other arguments as abcs_ida. */
abcs_status abcs_damp(abcs_handle* h, const int32_t* counts, const int64_t* offsets, const float* y,
                      int n_img, int H, int W, int B, int iters, double damping, int denoiser,
                      double lambda, const void* cnn_weights, const float* probe, float* x_out,
                      float* sigma_trace, float* alpha_trace, void* stream);

/* One image of an uneven batch (abcs_ida_batch). */
typedef struct abcs_image_desc {
    int32_t H, W, B;         /* image size in pixels, block size (4, 8, 16 or 32) */
    int32_t reserved;        /* 0 */
    int64_t block_offset;    /* index of the image's first block in counts / offsets */
    int64_t coeff_base;      /* added to the image's offsets to index y */
    int64_t pixel_offset;    /* index of the image's first pixel in x_out (dense Hc x Wc) */
} abcs_image_desc;

/* IDA (same iteration as abcs_ida) over a batch of images of different
 * sizes and block sizes, all iterations in ONE persistent cooperative
 * launch whose phases are separated by grid barriers (each wait bounded:
 * on expiry ABCS_DEV_TIMEOUT is set and the launch ends).  The launch is
 * captured once into a CUDA graph cached in the handle (keyed by all
 * arguments) and replayed; the denoiser tile height and CTAs per SM are
 * chosen the first time a batch shape is seen by timing each candidate on
 * the caller's data (autotuner; the choice is kept in the handle).
 *   desc        [host] n_img descriptors
 *   counts, offsets [device] blocks of image k at desc[k].block_offset ...;
 *               image k's coefficients at y[desc[k].coeff_base + offsets[.]]
 *   y           [device] float [y_len]
 *   x_out       [device] float, image k at x_out + desc[k].pixel_offset
 *   sigma_trace [device] float [n_img][iters] or NULL
 * denoiser: ABCS_DEN_NONE or ABCS_DEN_TIDCT (the learned denoiser runs
 * through abcs_ida). */
abcs_status abcs_ida_batch(abcs_handle* h, const abcs_image_desc* desc, int n_img, const int32_t* counts,
                           const int64_t* offsets, const float* y, int64_t y_len, int iters,
                           double damping, int denoiser, double lambda, float* x_out,
                           float* sigma_trace, void* stream);

/* The denoiser input of one IDA iteration: runs iterations 0 .. t-1 as
 * abcs_ida does, then the linear part of iteration t, and returns
 * r^t = x^t + A^T z^t (r_out [device] float [n_img][Hc][Wc]) and sigma^t
 * (sigma_out [device] float [n_img]).  Used to build training pairs
 * (r^t, clean image) for the learned denoiser. */
abcs_status abcs_ida_capture(abcs_handle* h, const int32_t* counts, const int64_t* offsets,
                             const float* y, int n_img, int H, int W, int B, int t, double damping,
                             int denoiser, double lambda, const void* cnn_weights, float* r_out,
                             float* sigma_out, void* stream);

/* The plain denoiser alone: for every image k, out = TI-DCT(in, lambda * sigma[k]).
 *   in, out [device] float [n_img][H][W] (dense, H, W >= 1; in != out)
 *   sigma   [device] float [n_img] */
abcs_status abcs_denoise_tidct(abcs_handle* h, const float* in, int n_img, int H, int W,
                               const float* sigma, double lambda, float* out, void* stream);

/* BM3D's hard-thresholding step (Dabov et al., ref. [22] of the paper; the
 * plain denoiser it pairs with IDA in Sec. VII) applied to every image:
 *   8 x 8 reference patches every 3 pixels (and at the last row / column);
 *   block matching over every position within 19 pixels, distance
 *   ||P_ref - P||^2 / 64, threshold tau = 2500 (sigma <= 40) or 5000;
 *   groups of the reference and its closest matches, at most 16, a power of
 *   two, ties in (distance, row, column) order;
 *   2D DCT of each patch, orthonormal Haar along the group, coefficients with
 *   |c| <= lambda sigma zeroed (the 3D DC kept), inverse transforms;
 *   aggregation weighted by 1 / (kept coefficients) and an 8 x 8 Kaiser
 *   window (beta 2).  BM3D uses lambda = 2.7.
 *   in, out [device] float [n_img][H][W] (in != out), H, W >= 8;
 *   sigma [device] float [n_img].
 * Uses the handle's workspace (two planes of the batch's size).  The
 * aggregation uses atomic adds, so results may differ in the last bits
 * between runs. */
abcs_status abcs_denoise_bm3d(abcs_handle* h, const float* in, int n_img, int H, int W, const float* sigma,
                              double lambda, float* out, void* stream);

/* Learned denoiser.  The paper plugs a pretrained 17-layer DnCNN into IDA
 * (Sec. VI-4); this library's learned denoiser is a smaller residual CNN of
 * the same kind, trained with the calls below:
 *   conv3x3 4->32 + ReLU, 6 x [conv3x3 32->32 + ReLU], conv3x3 32->1,
 *   x_hat = r - 255 * net(r / 255, sigma / 255, d, tau)   (zero 'same' padding),
 *   d = the measured fraction m_i / B^2 of the pixel's block (abcs_density_map;
 *   abcs_ida builds it from the counts; NULL means d = 0),
 *   tau = the iteration input, constant per image: abcs_ida and abcs_damp
 *   pass tau = min(t, 8) / 8 in iteration t (0 for the first denoising of
 *   A^T y); the calls below take it per image (NULL means 0).
 * Parameters are one FP32 vector of abcs_cnn_param_count() values, layer by
 * layer: w_l[co][ci][3][3] then b_l[co].  Inference runs from a packed
 * device copy (BF16 mid-layer weights) of abcs_cnn_packed_bytes() bytes. */
int64_t abcs_cnn_param_count(void);
size_t abcs_cnn_packed_bytes(void);

/* packed [device] <- params [device] (FP32 vector above). */
abcs_status abcs_cnn_pack(abcs_handle* h, const float* params, void* packed, void* stream);

/* out = x_hat(in, sigma[k], density, tau[k]) for every image k; in, out
 * [device] float [n_img][H][W] (in != out), sigma [device] float [n_img],
 * density [device] float [n_img][H][W] or NULL, tau [device] float [n_img]
 * or NULL. */
abcs_status abcs_cnn_denoise(abcs_handle* h, const void* packed, const float* in, const float* sigma,
                             const float* density, const float* tau, int n_img, int H, int W, float* out,
                             void* stream);

/* Loss L = mean((x_hat - clean)^2) / 255^2 over the n crops and its
 * gradient with respect to the parameters of `packed`.
 *   r, clean [device] float [n][H][W]; sigma [device] float [n]
 *   density [device] float [n][H][W] or NULL; tau [device] float [n] or NULL
 *   grad [device] float [abcs_cnn_param_count()]; loss [device] float [1] */
abcs_status abcs_cnn_grad(abcs_handle* h, const void* packed, const float* r, const float* clean,
                          const float* sigma, const float* density, const float* tau, int n, int H, int W,
                          float* grad, float* loss, void* stream);

/* One Adam step (beta = 0.9 / 0.999, eps = 1e-8, bias-corrected, `step`
 * counted from 1) on params [device] with moments adam_m, adam_v [device]
 * (same length, zero before step 1): packs params into `packed`, computes
 * the gradient of the batch, updates params and the moments, re-packs. */
abcs_status abcs_cnn_train_step(abcs_handle* h, float* params, float* adam_m, float* adam_v, int step,
                                double lr, void* packed, const float* r, const float* clean,
                                const float* sigma, const float* density, const float* tau, int n, int H,
                                int W, float* loss, void* stream);

/* Per-pixel measured fraction of the block (the learned denoiser's third
 * input): out[k][y][x] = counts[k n_B + (y / B) nbw + x / B] / B^2 over the
 * cropped Hc x Wc image.  counts [device] int32 [n_img * n_B] as written by
 * abcs_sense; out [device] float [n_img][Hc][Wc]. */
abcs_status abcs_density_map(abcs_handle* h, const int32_t* counts, int n_img, int H, int W, int B,
                             float* out, void* stream);

/* THI (Sec. IV; Sec. V-B, Table 2): full sensing with one threshold for the
 * whole image.  Per image, keep the M coefficients of largest magnitude,
 * irrespective of their block (by Parseval they carry the most energy, so
 * THI bounds what any adaptive per-block allocation can reach), and count
 * how many each block keeps.
 *   coeffs     [device] float [n_img][n_B][B*B]: every coefficient of every
 *              block of the cropped image, each block in zigzag-rank order
 *              (what abcs_sense writes with ABCS_ZZ at subrate 1).
 *   M          coefficients kept per image, 1 <= M <= n_B B^2.
 *   adaptive   [device] int32 [n_img * n_B] counts to correlate with (the
 *              counts abcs_sense writes for BBV or DD), or NULL.
 *   thi_counts [device] int32 [n_img * n_B] out: kept coefficients per block.
 *   rho        [device] double [n_img] out, or NULL (needs adaptive): the
 *              correlation coefficient of thi_counts and adaptive over the
 *              image's blocks, from exact integer sums; 0 when either
 *              sequence is constant.
 *   masked     [device] float, the layout of coeffs, out, or NULL: the kept
 *              coefficients, zeros elsewhere (abcs_reconstruct with counts
 *              B^2 then gives the THI image).
 * The magnitudes are ranked as the FP32 values given.  Among equal
 * magnitudes the lower (block, zigzag rank) index is kept first, so exactly
 * M coefficients are kept.  A NaN coefficient sets ABCS_DEV_NONFINITE.
 * Uses the handle's workspace (reallocated when too small). */
abcs_status abcs_thi(abcs_handle* h, const float* coeffs, int n_img, int H, int W, int B, int64_t M,
                     const int32_t* adaptive, int32_t* thi_counts, double* rho, float* masked, void* stream);

/* abcs_sense without any device allocation (the paper has no counterpart;
 * this is a library service).  For callers that may not call cudaMalloc
 * while running: a sensing loop whose device memory is reserved once at
 * start-up, or a real-time loop that cannot afford cudaMalloc's implicit
 * device synchronisation.  The arguments and results are those of
 * abcs_sense, with two differences: there is no handle, and only
 * precision ABCS_FP32 is built (a tensor-core precision returns
 * ABCS_ERR_UNSUPPORTED, a value outside abcs_precision ABCS_ERR_INVALID_ARG).
 * The scratch lives in one static device array of 4,784,640 bytes that
 * every GPU loading the library holds until the process exits.
 * Limits: n_img <= 4096 and n_img * n_B < 2^31 (else ABCS_ERR_INVALID_ARG);
 * n_img * n_B <= 1,048,576 blocks unless `pilot` is given, and at most
 * 65,536 pilot partial sums (n_img * ceil(n_B / 256) for BBV,
 * n_img * nbh * ceil(nbw * B / 256) for DD) (else ABCS_ERR_CAPACITY).
 * The first call on a device, with that device current, uploads the
 * transform tables, looks up the array's device address and clears its
 * status word; make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (e.g. on two streams)
 * race; serialise them.  Device status bits of these calls (an undecidable
 * DD decision, a bad count) collect in the array's status word until
 * abcs_sense_noalloc_status reads them. */
abcs_status abcs_sense_noalloc(const uint8_t* img, int n_img, int H, int W, int64_t pitch,
                               int64_t img_stride, int B, double subrate, int variant,
                               int precision, int32_t* counts, int64_t* offsets, float* coeffs,
                               int64_t coeff_capacity, int32_t* pilot, void* stream);

/* Wait for `stream`, then read and clear the device status word that the
 * abcs_sense_noalloc calls on the current device have set (no allocation).
 * Returns ABCS_OK if no bit was set, else ABCS_ERR_DEVICE with the bits
 * (ABCS_DEV_*) in *bits (bits may be NULL); ABCS_ERR_INVALID_ARG before the
 * first abcs_sense_noalloc call on the device.  Failure-detection test
 * hook, read on the host at each abcs_sense_noalloc call:
 * ABCS_FAULT_NOALLOC_BITS=n ORs the bits n into the word after the call's
 * kernels. */
abcs_status abcs_sense_noalloc_status(void* stream, uint32_t* bits);

/* Wait for `stream`, read and clear the device status word.  Returns
 * ABCS_OK if no bit was set, else ABCS_ERR_DEVICE with the bits in *bits
 * (bits may be NULL). */
abcs_status abcs_sync_status(abcs_handle* h, void* stream, uint32_t* bits);

#ifdef __cplusplus
}
#endif
#endif /* ABCS_H */
