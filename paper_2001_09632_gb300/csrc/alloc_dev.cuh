// Per-block measurement allocation, Eqs. 22-23, with the cap and
// redistribution rule of Sec. V-A, then the exclusive prefix (offsets) and
// the image bases of the batch.  Exact 64-bit integer arithmetic.
// Device functions shared by the stand-alone allocation kernel and by the
// pilot kernels, whose last CTA of an image allocates that image.
#pragma once
#include "abcs_common.cuh"

namespace abcs {

struct AllocParams {
    int mode;          // 0: every block gets m_fixed; 1: proportional to w
    int64_t R;         // phase-2 budget
    int cap;           // cap of m_i^2
    int m_add;         // added to every count (DD: m1)
    int m_fixed;       // mode 0 count of m_i^2 (ZZ / BBV with n_S = 0)
    int m_fallback;    // m_i^2 when sum w = 0 (BBV: floor(B^2 r), DD: m1)
};

// mode: 0 = ZZ (fixed m_zz), 1 = BBV, 2 = DD, 3 = BBV with n_S = 0 (fixed m_zz)
ABCS_HD AllocParams alloc_params(const SenseArgs& a, int mode) {
    AllocParams p{};
    p.cap = a.cap;
    p.R = a.R;
    if (mode == 0 || mode == 3) {
        p.mode = 0;
        p.m_fixed = a.m_zz;
    } else if (mode == 1) {
        p.mode = 1;
        p.m_fallback = a.m_zz;
    } else {
        p.mode = 1;
        p.m_add = a.m1;
        p.m_fallback = a.m1;
    }
    return p;
}

// Exclusive prefix over the CTA (blockDim.x a multiple of 32, <= 1024);
// `sh` holds 33 values; *total receives the CTA sum.
ABCS_D int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int64_t s = (lane < nw) ? sh[lane] : 0;
        int64_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < nw) sh[lane] = si - s;       // exclusive prefix of warp totals
        if (lane == nw - 1) sh[32] = si;        // CTA total
    }
    __syncthreads();
    *total = sh[32];
    return sh[wid] + incl - v;
}

// Counts and image-local offsets of image k, computed by the calling CTA.
// w: pilot values of the image's blocks; wpart: the image's cpi partial
// sums of w (both possibly written by other CTAs of the same kernel, so read
// through L2).  Writes counts, offsets and img_total[k].
ABCS_D void alloc_image(const int32_t* w, const unsigned long long* wpart, int cpi, int64_t nB,
                        const AllocParams& p, int k, int32_t* counts, int64_t* offsets, int64_t* img_total,
                        int64_t* sh, int64_t* sW) {
    const int32_t* wk = w + (int64_t)k * nB;
    int32_t* ck = counts + (int64_t)k * nB;
    int64_t* ok = offsets + (int64_t)k * nB;
    const int t = threadIdx.x, nt = blockDim.x;
    if (t < 32) {     // sum of the pilot CTAs' partials, fixed order
        unsigned long long v = 0;
        if (p.mode == 1)
            for (int j = t; j < cpi; j += 32) v += __ldcg(wpart + (int64_t)k * cpi + j);
        v = warp_sum(v);
        if (t == 0) *sW = (int64_t)v;
    }
    __syncthreads();
    const int64_t W = *sW;

    if (p.mode == 0 || W == 0) {
        const int m = p.m_add + (p.mode == 0 ? p.m_fixed : p.m_fallback);
        for (int64_t i = t; i < nB; i += nt) ck[i] = m;
    } else {
        // Eq. 22 / 23: m2 = floor(R w_i / W), capped; E = excess cut off
        int64_t E = 0;
        for (int64_t i = t; i < nB; i += nt) {
            int64_t a = p.R * (int64_t)__ldcg(wk + i) / W;
            if (a > p.cap) { E += a - p.cap; a = p.cap; }
            ck[i] = (int32_t)a;
        }
        E = block_sum(E, sh);
        // Sec. V-A: hand the excess to the blocks that are not fully measured,
        // in proportion to w, until nothing is left or nothing moves.
        for (int64_t round = 0; E > 0 && round <= nB + 1; ++round) {
            int64_t wu = 0;
            for (int64_t i = t; i < nB; i += nt) {
                const int32_t wi = __ldcg(wk + i);
                if (ck[i] < p.cap && wi > 0) wu += wi;
            }
            const int64_t WU = block_sum(wu, sh);
            if (WU == 0) break;
            int64_t added = 0, e2 = 0;
            for (int64_t i = t; i < nB; i += nt) {
                const int32_t wi = __ldcg(wk + i);
                if (ck[i] < p.cap && wi > 0) {
                    const int64_t add = E * (int64_t)wi / WU;
                    int64_t v = ck[i] + add;
                    added += add;
                    if (v > p.cap) { e2 += v - p.cap; v = p.cap; }
                    ck[i] = (int32_t)v;
                }
            }
            added = block_sum(added, sh);
            e2 = block_sum(e2, sh);
            if (added == 0) break;
            E = e2;
        }
        if (p.m_add)
            for (int64_t i = t; i < nB; i += nt) ck[i] += p.m_add;
    }
    __syncthreads();
    // exclusive prefix over contiguous chunks
    const int64_t chunk = (nB + nt - 1) / nt;
    const int64_t i0 = min(nB, (int64_t)t * chunk), i1 = min(nB, i0 + chunk);
    int64_t local = 0;
    for (int64_t i = i0; i < i1; ++i) local += ck[i];
    int64_t total;
    int64_t run = block_exclusive_scan(local, sh, &total);
    for (int64_t i = i0; i < i1; ++i) {
        ok[i] = run;
        run += ck[i];
    }
    if (t == 0) img_total[k] = total;
}

// After alloc_image: the last of the n allocating CTAs (counter `done`,
// reset by it) turns the per-image totals into image bases, an exclusive
// prefix with n + 1 entries.  No CTA waits for another.
ABCS_D void alloc_finish(int n, const int64_t* img_total, int64_t* img_base, unsigned* done, int64_t* sh,
                         bool* s_last) {
    const int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) {
        __threadfence();
        *s_last = atomicAdd(done, 1u) == (unsigned)n - 1;
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    const int chunk = (n + nt - 1) / nt;
    const int j0 = min(n, t * chunk), j1 = min(n, j0 + chunk);
    int64_t loc = 0;
    for (int j = j0; j < j1; ++j) loc += __ldcg(img_total + j);
    int64_t tot;
    int64_t base = block_exclusive_scan(loc, sh, &tot);
    for (int j = j0; j < j1; ++j) {
        img_base[j] = base;
        base += __ldcg(img_total + j);
    }
    if (t == 0) {
        img_base[n] = tot;
        *done = 0u;
    }
}

// Fused tail of a pilot kernel whose CTAs of image k number `cpi`: the last
// of them (per-image counter img_done[k], reset by it) allocates image k;
// the last image allocated computes the image bases.
ABCS_D void pilot_alloc_tail(const SenseArgs& a, int mode, int k, int cpi, int64_t* sh, int64_t* sW,
                             bool* s_last) {
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(a.img_done + k, 1u) == (unsigned)cpi - 1;
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.img_done[k] = 0u;
    alloc_image(a.w, a.wpart, cpi, a.g.n_blocks, alloc_params(a, mode), k, a.counts, a.offsets, a.img_total, sh,
                sW);
    if (a.pilot_bases) alloc_finish(a.g.n_img, a.img_total, a.img_base, a.done, sh, s_last);
}

}  // namespace abcs
