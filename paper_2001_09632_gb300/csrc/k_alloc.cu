// Stand-alone allocation kernel (Eqs. 22-23 and Sec. V-A): one CTA per
// image; the last CTA writes the image bases (unless the sensing kernel
// derives them).  Used when there is no pilot
// (L-DCT-ZZ, BBV with n_S = 0) and by the allocation-free sensing entry
// point; otherwise the pilot kernels allocate in their fused tail.
#include "alloc_dev.cuh"

namespace abcs {

namespace {

constexpr int kAllocThreads = 1024;

__global__ void __launch_bounds__(kAllocThreads)
alloc_kernel(const int32_t* __restrict__ w, const unsigned long long* __restrict__ wpart, int cpi, int64_t nB,
             AllocParams p, int32_t* __restrict__ counts, int64_t* __restrict__ offsets,
             int64_t* __restrict__ img_total, int64_t* __restrict__ img_base, unsigned* done, int bases) {
    __shared__ int64_t sh[33];
    __shared__ int64_t sW;
    __shared__ bool s_last;
    griddep_wait();
    alloc_image(w, wpart, cpi, nB, p, blockIdx.x, counts, offsets, img_total, sh, &sW);
    if (bases) alloc_finish(gridDim.x, img_total, img_base, done, sh, &s_last);
}

}  // namespace

cudaError_t launch_allocate(const SenseArgs& a, int mode, cudaStream_t s) {
    return launch_pdl(alloc_kernel, dim3(a.g.n_img), dim3(kAllocThreads), 0, s, (const int32_t*)a.w,
                      (const unsigned long long*)a.wpart, a.pilot_cpi, (int64_t)a.g.n_blocks, alloc_params(a, mode),
                      a.counts, a.offsets, a.img_total, a.img_base, a.done, a.pilot_bases);
}

}  // namespace abcs
