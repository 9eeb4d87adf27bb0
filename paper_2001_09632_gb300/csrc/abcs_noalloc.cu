// abcs_sense_noalloc: sensing for callers that cannot allocate device memory.
//
// Some callers of this library are not allowed to call cudaMalloc once they
// are running: a sensor pipeline with a fixed device-memory budget that is
// reserved up front, or a real-time loop in which the implicit device-wide
// synchronisation and unbounded latency of cudaMalloc/cudaFree would break
// the frame deadline.  abcs_sense keeps its scratch (per-block pilot values,
// per-image sums) in a handle workspace that grows with cudaMalloc; this
// entry point keeps the same scratch in one fixed, file-scope device array
// instead, so a call allocates nothing.  The caller still provides the
// image and every output buffer.
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "abcs_common.cuh"

namespace abcs {
abcs_status record_error(abcs_status s, const char* msg);
}

namespace {

using namespace abcs;

// Limits of the static scratch.
constexpr int kNoAllocMaxImages = 4096;          // images per call
constexpr int64_t kNoAllocMaxBlocks = 1 << 20;   // blocks per call when pilot == NULL
constexpr int64_t kNoAllocMaxParts = 1 << 16;    // pilot partial sums per call
constexpr size_t kOffStatus = 0;                 // status word, allocation CTA counter
constexpr size_t kOffTotal = 256;
constexpr size_t kOffBase = kOffTotal + 8 * (size_t)kNoAllocMaxImages;
constexpr size_t kOffPart = (kOffBase + 8 * (size_t)(kNoAllocMaxImages + 1) + 255) / 256 * 256;
constexpr size_t kOffW = kOffPart + 8 * (size_t)kNoAllocMaxParts;
constexpr size_t kScratchBytes = kOffW + 4 * (size_t)kNoAllocMaxBlocks;   // 4,784,640 bytes

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void or_status_kernel(uint32_t* st, uint32_t bits) { set_status(st, bits); }

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[kMaxDevices];       // device address of the array, per device

abcs_status err(abcs_status s, const char* fmt, long long a = 0, long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    return record_error(s, buf);
}

// Once per device, with that device current: upload the transform tables
// and look up the device address of the scratch array.
abcs_status setup_device(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_dev[dev]) {
        *out = g_scratch_dev[dev];
        return ABCS_OK;
    }
    cudaError_t e = upload_tables_pilot();
    if (e == cudaSuccess) e = upload_tables_dct();
    if (e != cudaSuccess) return record_error(ABCS_ERR_CUDA, cudaGetErrorString(e));
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return record_error(ABCS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    // the status word accumulates the device bits of every call until
    // abcs_sense_noalloc_status reads and clears it: start it at zero once
    e = cudaMemset(p, 0, 2 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return record_error(ABCS_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    *out = g_scratch_dev[dev];
    return ABCS_OK;
}

// The scratch array of the current device, set up by an earlier call.
unsigned char* current_scratch(int* dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    *dev_out = dev;
    return g_scratch_dev[dev];
}

}  // namespace

extern "C" abcs_status abcs_sense_noalloc(const uint8_t* img, int n_img, int H, int W,
                                          int64_t pitch, int64_t img_stride, int B,
                                          double subrate, int variant, int precision,
                                          int32_t* counts, int64_t* offsets, float* coeffs,
                                          int64_t coeff_capacity, int32_t* pilot, void* stream) {
    abcs_plan_info p;
    abcs_status st = abcs_plan(H, W, B, subrate, variant, &p);
    if (st) return st;
    if (n_img < 1 || n_img > kNoAllocMaxImages)
        return err(ABCS_ERR_INVALID_ARG, "n_img must be in [1, %lld] for abcs_sense_noalloc",
                   kNoAllocMaxImages);
    if (precision < ABCS_FP32 || precision > ABCS_TC_BF16)
        return err(ABCS_ERR_INVALID_ARG, "bad precision %lld", precision);
    if (precision != ABCS_FP32)
        return err(ABCS_ERR_UNSUPPORTED,
                   "abcs_sense_noalloc computes in FP32 only (precision %lld requested)", precision);
    const int64_t nb_all = (int64_t)n_img * p.n_blocks;
    if (nb_all >= (1LL << 31)) return err(ABCS_ERR_INVALID_ARG, "more than 2^31 - 1 blocks in one call");
    if (!pilot && nb_all > kNoAllocMaxBlocks)
        return err(ABCS_ERR_CAPACITY,
                   "abcs_sense_noalloc: %lld blocks exceed the static scratch limit of %lld "
                   "(pass a pilot buffer to lift it)", nb_all, kNoAllocMaxBlocks);
    SenseArgs a{};
    a.g.n_img = n_img; a.g.H = H; a.g.W = W; a.g.B = B;
    a.g.nbh = H / B; a.g.nbw = W / B;
    a.g.Hc = a.g.nbh * B; a.g.Wc = a.g.nbw * B;
    a.g.n_blocks = p.n_blocks;
    a.g.pitch = pitch; a.g.img_stride = img_stride;
    a.variant = variant;
    a.pilot_cpi = pilot_ctas_per_image(a);
    if ((int64_t)n_img * a.pilot_cpi > kNoAllocMaxParts)
        return err(ABCS_ERR_CAPACITY,
                   "abcs_sense_noalloc: %lld pilot partial sums exceed the static scratch limit of %lld",
                   (int64_t)n_img * a.pilot_cpi, kNoAllocMaxParts);
    if (!img || !counts || !offsets || !coeffs) return err(ABCS_ERR_INVALID_ARG, "NULL buffer");
    if (pitch < W) return err(ABCS_ERR_INVALID_ARG, "pitch %lld < W %lld", pitch, W);
    if (n_img > 1 && img_stride < pitch * H)
        return err(ABCS_ERR_INVALID_ARG, "img_stride smaller than pitch * H");
    if (coeff_capacity < (int64_t)n_img * p.M)
        return err(ABCS_ERR_CAPACITY, "coeff_capacity %lld < n_img * M = %lld", coeff_capacity,
                   (int64_t)n_img * p.M);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(ABCS_ERR_CUDA, "no usable current CUDA device");
    unsigned char* scratch = nullptr;
    st = setup_device(dev, &scratch);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    a.img = img;
    a.precision = precision;
    a.L = p.L; a.X0 = p.X0; a.nS = p.nS; a.m1 = p.m1; a.m_zz = p.m_zz; a.T = p.T; a.cap = p.cap;
    a.R = p.R;
    a.counts = counts;
    a.offsets = offsets;
    a.coeffs = coeffs;
    a.capacity = coeff_capacity;
    a.status = reinterpret_cast<uint32_t*>(scratch + kOffStatus);
    a.done = reinterpret_cast<unsigned*>(scratch + kOffStatus) + 1;
    a.img_total = reinterpret_cast<int64_t*>(scratch + kOffTotal);
    a.img_base = reinterpret_cast<int64_t*>(scratch + kOffBase);
    a.wpart = reinterpret_cast<unsigned long long*>(scratch + kOffPart);
    a.w = pilot ? pilot : reinterpret_cast<int32_t*>(scratch + kOffW);
    a.pilot_bases = 1;

    // The array keeps the previous call's contents.  Pilot values, partial
    // sums, totals and bases are fully overwritten by every call; the
    // allocation CTA counter must start at zero.  The status word is left
    // as it is: it collects the bits of every call until it is read.
    cudaError_t e = cudaMemsetAsync(a.done, 0, sizeof(uint32_t), s);
    int mode = 0;
    if (e == cudaSuccess) {
        if (variant == ABCS_BBV && p.nS > 0) {
            e = launch_bbv_pilot(a, s);
            mode = 1;
        } else if (variant == ABCS_DD) {
            e = launch_dd_pilot(a, s);
            mode = 2;
        } else {
            mode = (variant == ABCS_BBV) ? 3 : 0;
            if (pilot) e = cudaMemsetAsync(pilot, 0, nb_all * sizeof(int32_t), s);
        }
    }
    if (e == cudaSuccess) e = launch_allocate(a, mode, s);
    if (e == cudaSuccess) e = launch_sense_pack(a, s);
    // Failure-detection test hook (host side): ABCS_FAULT_NOALLOC_BITS=n ORs
    // the bits n into the status word after the call's kernels, as a device
    // condition (an undecidable DD tie, a bad count) would.
    if (e == cudaSuccess)
        if (const char* f = getenv("ABCS_FAULT_NOALLOC_BITS")) {
            or_status_kernel<<<1, 1, 0, s>>>(a.status, (uint32_t)strtoul(f, nullptr, 0));
            e = cudaGetLastError();
        }
    if (e != cudaSuccess) return record_error(ABCS_ERR_CUDA, cudaGetErrorString(e));
    return ABCS_OK;
}

extern "C" abcs_status abcs_sense_noalloc_status(void* stream, uint32_t* bits) {
    int dev = 0;
    unsigned char* scratch = current_scratch(&dev);
    if (bits) *bits = 0;
    if (!scratch)
        return err(ABCS_ERR_INVALID_ARG,
                   "abcs_sense_noalloc_status: no abcs_sense_noalloc call on the current device yet");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    uint32_t v = 0;
    // a plain copy into a host variable and a memset: neither allocates
    if (e == cudaSuccess) e = cudaMemcpy(&v, scratch + kOffStatus, sizeof v, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(scratch + kOffStatus, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return record_error(ABCS_ERR_CUDA, cudaGetErrorString(e));
    if (bits) *bits = v;
    if (v) return err(ABCS_ERR_DEVICE, "device status bits 0x%llx", (long long)v);
    return ABCS_OK;
}
