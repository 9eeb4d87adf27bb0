// THI (Sec. IV; Sec. V-B and Table 2): with every DCT coefficient sensed,
// keep per image the M coefficients of largest magnitude, irrespective of
// their block, and report how many each block keeps.
//
// Keys are the bit patterns of |c| (FP32, non-negative, so unsigned order
// is magnitude order).  Four radix-select passes of 8 bits find, per image,
// the key t of the M-th largest coefficient and how many of the
// coefficients equal to t are kept (what is left of M after those above t).
// Per block: gt = #{key > t}, eq = #{key == t}; the ties are kept in
// (block, zigzag rank) order, so exactly M coefficients are kept.
#include "abcs_common.cuh"
#include "alloc_dev.cuh"

namespace abcs {

namespace {

ABCS_D uint32_t thi_key(float c) { return __float_as_uint(c) & 0x7FFFFFFFu; }

// rem[k] = M (the rank sought), histograms cleared
__global__ void __launch_bounds__(256) thi_init_kernel(int64_t M, int64_t* __restrict__ rem, uint32_t* __restrict__ hist) {
    griddep_wait();
    hist[(int64_t)blockIdx.x * 256 + threadIdx.x] = 0u;
    if (threadIdx.x == 0) rem[blockIdx.x] = M;
}

// Pass p: per-image histogram of key digit (24 - 8p) over the keys whose
// higher digits equal prefix[k].  Grid (chunks, images).
__global__ void __launch_bounds__(256) thi_hist_kernel(const float* __restrict__ c, int64_t per_img, int pass,
                                                       const uint32_t* __restrict__ prefix,
                                                       uint32_t* __restrict__ hist, uint32_t* status) {
    __shared__ uint32_t h[256];
    griddep_wait();
    const int k = blockIdx.y;
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int shift = 24 - 8 * pass;
    const uint32_t pre = pass ? prefix[k] : 0u;
    const uint32_t hmask = pass ? (0xFFFFFFFFu << (shift + 8)) : 0u;
    const float4* ck = reinterpret_cast<const float4*>(c + (int64_t)k * per_img);   // per_img % 16 == 0
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_img / 4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(ck + i);
        const uint32_t kk[4] = {thi_key(v.x), thi_key(v.y), thi_key(v.z), thi_key(v.w)};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            bad |= kk[e] > 0x7F800000u;                                  // NaN
            if ((kk[e] & hmask) == pre) atomicAdd(&h[(kk[e] >> shift) & 255u], 1u);
        }
    }
    if (pass == 0 && bad) set_status(status, ABCS_DEV_NONFINITE);
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + (int64_t)k * 256 + threadIdx.x, h[threadIdx.x]);
}

// One CTA of 256 threads per image: the digit that holds the rem-th largest
// matching key; rem becomes its rank among the keys with that digit.  The
// histogram is cleared for the next pass.
__global__ void __launch_bounds__(256) thi_pick_kernel(int pass, uint32_t* __restrict__ prefix,
                                                       int64_t* __restrict__ rem, uint32_t* __restrict__ hist) {
    griddep_wait();
    const int k = blockIdx.x, t = threadIdx.x;
    __shared__ unsigned long long warp_tot[8];
    const unsigned hv = hist[(int64_t)k * 256 + t];
    hist[(int64_t)k * 256 + t] = 0u;
    // suffix sums: above(d) = sum of bins > d; digit d holds the rem-th largest key
    // when above(d) < rem <= above(d) + h[d] (digit 0 if none above)
    const int lane = t & 31, warp = t >> 5;
    unsigned long long incl = hv;                                   // within the warp, from higher digits down
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += v;
    }
    if (lane == 0) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long higher = 0;
    for (int w = warp + 1; w < 8; ++w) higher += warp_tot[w];
    const unsigned long long above = incl - hv + higher;           // bins > t
    const int64_t r = rem[k];
    __syncthreads();                                                // every thread has read rem[k]
    const bool here = (int64_t)above < r && (r <= (int64_t)(above + hv) || t == 0);
    if (here) {
        rem[k] = r - (int64_t)above;
        prefix[k] = (pass ? prefix[k] : 0u) | ((uint32_t)t << (24 - 8 * pass));
    }
}

// One warp per block: gt_b = #{key > t}, eq_b = #{key == t}.
__global__ void __launch_bounds__(256) thi_count_kernel(const float* __restrict__ c, int64_t nblk, int bb, int nB,
                                                        const uint32_t* __restrict__ prefix, int32_t* __restrict__ gt,
                                                        int32_t* __restrict__ eq) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nblk;
         b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t t = __ldg(prefix + b / nB);
        const float* cb = c + b * bb;
        int g = 0, e = 0;
        for (int j = lane; j < bb; j += 32) {
            const uint32_t key = thi_key(__ldg(cb + j));
            g += key > t;
            e += key == t;
        }
        g = warp_sum(g);
        e = warp_sum(e);
        if (lane == 0) {
            gt[b] = g;
            eq[b] = e;
        }
    }
}

// One CTA (1024 threads) per image: ties kept in block order
// (taken_b = clamp(need - ties before b, 0, eq_b)), counts gt_b + taken_b,
// and with `adaptive` the correlation coefficient of the two count
// sequences from exact 64-bit sums.  taken_b overwrites eq_b.
__global__ void __launch_bounds__(1024) thi_finish_kernel(int nB, const int64_t* __restrict__ rem,
                                                          const int32_t* __restrict__ gt, int32_t* __restrict__ eq,
                                                          int32_t* __restrict__ counts,
                                                          const int32_t* __restrict__ adaptive,
                                                          double* __restrict__ rho) {
    __shared__ int64_t sh[33];
    griddep_wait();
    const int k = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
    const int64_t base = (int64_t)k * nB;
    const int chunk = (nB + nt - 1) / nt;
    const int i0 = min(nB, t * chunk), i1 = min(nB, i0 + chunk);
    int64_t loc = 0;
    for (int i = i0; i < i1; ++i) loc += eq[base + i];
    int64_t tot;
    int64_t before = block_exclusive_scan(loc, sh, &tot);
    const int64_t need = rem[k];
    int64_t sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    for (int i = i0; i < i1; ++i) {
        const int64_t e = eq[base + i];
        int64_t take = need - before;
        take = take < 0 ? 0 : (take > e ? e : take);
        before += e;
        const int64_t x = gt[base + i] + take;
        counts[base + i] = (int32_t)x;
        eq[base + i] = (int32_t)take;
        if (adaptive) {
            const int64_t y = __ldg(adaptive + base + i);
            sx += x;
            sy += y;
            sxx += x * x;
            syy += y * y;
            sxy += x * y;
        }
    }
    if (!adaptive || !rho) return;
    sx = block_sum(sx, sh);
    sy = block_sum(sy, sh);
    sxx = block_sum(sxx, sh);
    syy = block_sum(syy, sh);
    sxy = block_sum(sxy, sh);
    if (t == 0) {
        const int64_t n = nB;
        const int64_t vx = n * sxx - sx * sx, vy = n * syy - sy * sy, cxy = n * sxy - sx * sy;
        rho[k] = (vx == 0 || vy == 0) ? 0.0 : (double)cxy / (sqrt((double)vx) * sqrt((double)vy));
    }
}

// One warp per block: the kept coefficients, zeros elsewhere.  Ties are
// kept in rank order: the j-th tie of the block (counted by ballot) is kept
// if j < taken_b.
__global__ void __launch_bounds__(256) thi_mask_kernel(const float* __restrict__ c, int64_t nblk, int bb, int nB,
                                                       const uint32_t* __restrict__ prefix,
                                                       const int32_t* __restrict__ taken, float* __restrict__ out) {
    griddep_wait();
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nblk;
         b += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint32_t t = __ldg(prefix + b / nB);
        const int tk = __ldg(taken + b);
        const float* cb = c + b * bb;
        float* ob = out + b * bb;
        int seen = 0;
        for (int j0 = 0; j0 < bb; j0 += 32) {
            const int j = j0 + lane;                                     // bb % 32 == 0 or bb == 16
            const bool in = j < bb;
            const float v = in ? __ldg(cb + j) : 0.f;
            const uint32_t key = thi_key(v);
            const uint32_t ties = __ballot_sync(0xffffffffu, in && key == t);
            const bool keep = key > t || (key == t && seen + __popc(ties & lt) < tk);
            if (in) ob[j] = keep ? v : 0.f;
            seen += __popc(ties);
        }
    }
}

}  // namespace

cudaError_t launch_thi(const float* coeffs, int n_img, int nB, int bb, int64_t M, const int32_t* adaptive,
                       int32_t* counts, double* rho, float* masked, uint32_t* prefix, int64_t* rem, uint32_t* hist,
                       int32_t* gt, int32_t* eq, uint32_t* status, cudaStream_t s) {
    const int64_t per_img = (int64_t)nB * bb, nblk = (int64_t)n_img * nB;
    int dev, sms;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = launch_pdl(thi_init_kernel, dim3((unsigned)n_img), dim3(256), 0, s, M, rem, hist);
    if (e) return e;
    // chunks per image: about eight CTAs per SM over the whole batch
    const int64_t want = ((int64_t)sms * 8 + n_img - 1) / n_img, cap = (per_img / 4 + 255) / 256;
    const unsigned chunks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    for (int pass = 0; pass < 4 && !e; ++pass) {
        e = launch_pdl(thi_hist_kernel, dim3(chunks, (unsigned)n_img), dim3(256), 0, s, coeffs, per_img, pass,
                       (const uint32_t*)prefix, hist, status);
        if (!e) e = launch_pdl(thi_pick_kernel, dim3((unsigned)n_img), dim3(256), 0, s, pass, prefix, rem, hist);
    }
    const unsigned gw = (unsigned)((nblk * 32 + 255) / 256 < (int64_t)sms * 16 ? (nblk * 32 + 255) / 256 : sms * 16);
    if (!e)
        e = launch_pdl(thi_count_kernel, dim3(gw), dim3(256), 0, s, coeffs, nblk, bb, nB, (const uint32_t*)prefix,
                       gt, eq);
    if (!e)
        e = launch_pdl(thi_finish_kernel, dim3((unsigned)n_img), dim3(1024), 0, s, nB, (const int64_t*)rem,
                       (const int32_t*)gt, eq, counts, adaptive, rho);
    if (!e && masked)
        e = launch_pdl(thi_mask_kernel, dim3(gw), dim3(256), 0, s, coeffs, nblk, bb, nB, (const uint32_t*)prefix,
                       (const int32_t*)eq, masked);
    return e;
}

}  // namespace abcs
