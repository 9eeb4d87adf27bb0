"""ctypes binding of libabcs.so (C ABI in include/abcs.h).

Every function here has the name of the C entry point it calls and does
argument marshalling only: torch tensors become device pointers, a torch
stream becomes a cudaStream_t, non-OK statuses become AbcsError.  All
compute happens in the library's CUDA kernels; there is no fallback, and
importing this module fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libabcs.so")

ZZ, BBV, DD = 0, 1, 2
FP32, TC_FP16X2, TC_BF16X2, TC_BF16 = 0, 1, 2, 3
DEN_NONE, DEN_TIDCT, DEN_CNN, DEN_BM3D = 0, 1, 2, 3
VARIANTS = {"zz": ZZ, "bbv": BBV, "dd": DD}
PRECISIONS = {"fp32": FP32, "fp16x2": TC_FP16X2, "bf16x2": TC_BF16X2, "bf16": TC_BF16}

DEV_CAPACITY, DEV_AMBIGUOUS, DEV_NONFINITE, DEV_TIMEOUT, DEV_BADCOUNT = 0x1, 0x2, 0x4, 0x8, 0x10

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CAPACITY", 4: "OOM", 5: "CUDA",
                6: "TIMEOUT", 7: "NONFINITE", 8: "DEVICE"}


class AbcsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ABCS_{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class abcs_image_desc(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("B", C.c_int32), ("reserved", C.c_int32),
                ("block_offset", C.c_int64), ("coeff_base", C.c_int64), ("pixel_offset", C.c_int64)]


class abcs_sense_desc(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("B", C.c_int32), ("variant", C.c_int32),
                ("subrate", C.c_double), ("img_offset", C.c_int64), ("pitch", C.c_int64)]


class abcs_plan_info(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("B", C.c_int32), ("variant", C.c_int32),
                ("nbh", C.c_int32), ("nbw", C.c_int32), ("n_blocks", C.c_int64), ("N", C.c_int64),
                ("M", C.c_int64), ("CF", C.c_double), ("L", C.c_int32), ("X0", C.c_int32),
                ("nS", C.c_int32), ("m1", C.c_int32), ("m_zz", C.c_int32), ("T", C.c_int32),
                ("cap", C.c_int32), ("M_bbv", C.c_int64), ("R", C.c_int64), ("max_coeffs", C.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built: run `python -m paper_2001_09632_gb300.build` "
                      "(there is no non-CUDA fallback)")
lib = C.CDLL(LIB_PATH)

_P, _I, _L, _D = C.c_void_p, C.c_int, C.c_int64, C.c_double
_SIGS = {
    "abcs_create": [C.POINTER(C.c_void_p)],
    "abcs_destroy": [_P],
    "abcs_last_error": [],
    "abcs_plan": [_I, _I, _I, _D, _I, C.POINTER(abcs_plan_info)],
    "abcs_sense": [_P, _P, _I, _I, _I, _L, _L, _I, _D, _I, _I, _P, _P, _P, _L, _P, _P],
    "abcs_sense_batch": [_P, _P, _P, _I, _I, _P, _P, _P, _L, _P, _P],
    "abcs_reconstruct": [_P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P, _P],
    "abcs_ida": [_P, _P, _P, _P, _I, _I, _I, _I, _I, _D, _I, _D, _P, _P, _P, _P],
    "abcs_denoise_tidct": [_P, _P, _I, _I, _I, _P, _D, _P, _P],
    "abcs_denoise_bm3d": [_P, _P, _I, _I, _I, _P, _D, _P, _P],
    "abcs_sync_status": [_P, _P, C.POINTER(C.c_uint32)],
    "abcs_set_ida_precision": [_P, _I],
    "abcs_psnr_ssim": [_P, _P, _P, _I, _I, _I, _L, _L, _P, _P, _P],
    "abcs_sense_noalloc": [_P, _I, _I, _I, _L, _L, _I, _D, _I, _I, _P, _P, _P, _L, _P, _P],
    "abcs_sense_noalloc_status": [_P, C.POINTER(C.c_uint32)],
    "abcs_ida_batch": [_P, _P, _I, _P, _P, _P, _L, _I, _D, _I, _D, _P, _P, _P],
    "abcs_ida_capture": [_P, _P, _P, _P, _I, _I, _I, _I, _I, _D, _I, _D, _P, _P, _P, _P],
    "abcs_cnn_param_count": [],
    "abcs_cnn_packed_bytes": [],
    "abcs_cnn_pack": [_P, _P, _P, _P],
    "abcs_cnn_denoise": [_P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P],
    "abcs_cnn_grad": [_P, _P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P, _P],
    "abcs_cnn_train_step": [_P, _P, _P, _P, _I, _D, _P, _P, _P, _P, _P, _P, _I, _I, _I, _P, _P],
    "abcs_density_map": [_P, _P, _I, _I, _I, _I, _P, _P],
    "abcs_thi": [_P, _P, _I, _I, _I, _I, C.c_int64, _P, _P, _P, _P, _P],
    "abcs_damp": [_P, _P, _P, _P, _I, _I, _I, _I, _I, C.c_double, _I, C.c_double, _P, _P, _P, _P, _P, _P],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = {"abcs_last_error": C.c_char_p, "abcs_destroy": None, "abcs_cnn_param_count": C.c_int64,
                  "abcs_cnn_packed_bytes": C.c_size_t}.get(_name, C.c_int)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int):
    if status != 0:
        raise AbcsError(status, lib.abcs_last_error().decode())


def abcs_last_error() -> str:
    return lib.abcs_last_error().decode()


def abcs_create() -> int:
    h = C.c_void_p()
    _check(lib.abcs_create(C.byref(h)))
    return h.value


def abcs_destroy(h: int) -> None:
    lib.abcs_destroy(h)


def abcs_plan(H: int, W: int, B: int, subrate: float, variant: int) -> dict:
    info = abcs_plan_info()
    _check(lib.abcs_plan(H, W, B, subrate, variant, C.byref(info)))
    return info.as_dict()


def abcs_sense(h, img, n_img, H, W, pitch, img_stride, B, subrate, variant, precision,
               counts, offsets, coeffs, coeff_capacity, pilot=None, stream=None) -> None:
    _check(lib.abcs_sense(h, _ptr(img), n_img, H, W, pitch, img_stride, B, subrate, variant,
                          precision, _ptr(counts), _ptr(offsets), _ptr(coeffs), coeff_capacity,
                          _ptr(pilot), _stream(stream)))


def abcs_sense_batch(h, img, descs, precision, counts, offsets, coeffs, coeff_capacity, pilot=None,
                     stream=None) -> None:
    """descs: list of (H, W, B, variant, subrate, img_offset, pitch)."""
    arr = (abcs_sense_desc * len(descs))(*[abcs_sense_desc(H, W, B, v, r, o, p) for (H, W, B, v, r, o, p) in descs])
    _check(lib.abcs_sense_batch(h, _ptr(img), arr, len(descs), precision, _ptr(counts), _ptr(offsets),
                                _ptr(coeffs), coeff_capacity, _ptr(pilot), _stream(stream)))


def abcs_reconstruct(h, counts, offsets, coeffs, n_img, H, W, B, precision, out=None, out_u8=None,
                     stream=None) -> None:
    _check(lib.abcs_reconstruct(h, _ptr(counts), _ptr(offsets), _ptr(coeffs), n_img, H, W, B,
                                precision, _ptr(out), _ptr(out_u8), _stream(stream)))


def abcs_ida(h, counts, offsets, y, n_img, H, W, B, iters, damping, denoiser, lam, cnn_weights,
             x_out, sigma_trace=None, stream=None) -> None:
    _check(lib.abcs_ida(h, _ptr(counts), _ptr(offsets), _ptr(y), n_img, H, W, B, iters, damping,
                        denoiser, lam, _ptr(cnn_weights), _ptr(x_out), _ptr(sigma_trace),
                        _stream(stream)))


def abcs_ida_batch(h, descs, counts, offsets, y, y_len, iters, damping, denoiser, lam, x_out,
                   sigma_trace=None, stream=None) -> None:
    """descs: list of (H, W, B, block_offset, coeff_base, pixel_offset)."""
    arr = (abcs_image_desc * len(descs))(*[abcs_image_desc(H, W, B, 0, bo, cb, po)
                                           for (H, W, B, bo, cb, po) in descs])
    _check(lib.abcs_ida_batch(h, arr, len(descs), _ptr(counts), _ptr(offsets), _ptr(y), y_len, iters,
                              damping, denoiser, lam, _ptr(x_out), _ptr(sigma_trace), _stream(stream)))


def abcs_ida_capture(h, counts, offsets, y, n_img, H, W, B, t, damping, denoiser, lam, cnn_weights,
                     r_out, sigma_out, stream=None) -> None:
    _check(lib.abcs_ida_capture(h, _ptr(counts), _ptr(offsets), _ptr(y), n_img, H, W, B, t, damping,
                                denoiser, lam, _ptr(cnn_weights), _ptr(r_out), _ptr(sigma_out),
                                _stream(stream)))


def abcs_denoise_bm3d(h, inp, n_img, H, W, sigma, lam, out, stream=None) -> None:
    """BM3D's hard-thresholding step (lam = lambda_3D, 2.7 in BM3D)."""
    _check(lib.abcs_denoise_bm3d(h, _ptr(inp), n_img, H, W, _ptr(sigma), lam, _ptr(out), _stream(stream)))


def abcs_denoise_tidct(h, inp, n_img, H, W, sigma, lam, out, stream=None) -> None:
    _check(lib.abcs_denoise_tidct(h, _ptr(inp), n_img, H, W, _ptr(sigma), lam, _ptr(out),
                                  _stream(stream)))


def abcs_sense_noalloc(img, n_img, H, W, pitch, img_stride, B, subrate, variant, precision,
                       counts, offsets, coeffs, coeff_capacity, pilot=None, stream=None) -> None:
    """abcs_sense with its scratch in a static device array (no allocation)."""
    _check(lib.abcs_sense_noalloc(_ptr(img), n_img, H, W, pitch, img_stride, B, subrate, variant,
                                  precision, _ptr(counts), _ptr(offsets), _ptr(coeffs),
                                  coeff_capacity, _ptr(pilot), _stream(stream)))


def abcs_sense_noalloc_status(stream=None) -> int:
    """Waits for the stream; returns and clears the device status bits of the
    abcs_sense_noalloc calls on the current device (0 = clean)."""
    bits = C.c_uint32(0)
    st = lib.abcs_sense_noalloc_status(_stream(stream), C.byref(bits))
    if st not in (0, 8):
        _check(st)
    return bits.value


def abcs_cnn_param_count() -> int:
    return lib.abcs_cnn_param_count()


def abcs_cnn_packed_bytes() -> int:
    return lib.abcs_cnn_packed_bytes()


def abcs_cnn_pack(h, params, packed, stream=None) -> None:
    _check(lib.abcs_cnn_pack(h, _ptr(params), _ptr(packed), _stream(stream)))


def abcs_cnn_denoise(h, packed, inp, sigma, density, n_img, H, W, out, stream=None, tau=None) -> None:
    """density: per-pixel measured fraction (abcs_density_map) or None;
    tau: the iteration input per image or None (0)."""
    _check(lib.abcs_cnn_denoise(h, _ptr(packed), _ptr(inp), _ptr(sigma), _ptr(density), _ptr(tau), n_img, H, W,
                                _ptr(out), _stream(stream)))


def abcs_cnn_grad(h, packed, r, clean, sigma, density, n, H, W, grad, loss, stream=None, tau=None) -> None:
    _check(lib.abcs_cnn_grad(h, _ptr(packed), _ptr(r), _ptr(clean), _ptr(sigma), _ptr(density), _ptr(tau), n, H,
                             W, _ptr(grad), _ptr(loss), _stream(stream)))


def abcs_cnn_train_step(h, params, adam_m, adam_v, step, lr, packed, r, clean, sigma, density, n, H, W, loss,
                        stream=None, tau=None) -> None:
    _check(lib.abcs_cnn_train_step(h, _ptr(params), _ptr(adam_m), _ptr(adam_v), step, lr, _ptr(packed),
                                   _ptr(r), _ptr(clean), _ptr(sigma), _ptr(density), _ptr(tau), n, H, W,
                                   _ptr(loss), _stream(stream)))


def abcs_density_map(h, counts, n_img, H, W, B, out, stream=None) -> None:
    """out[k][y][x] = m_i / B^2 of the block holding pixel (y, x)."""
    _check(lib.abcs_density_map(h, _ptr(counts), n_img, H, W, B, _ptr(out), _stream(stream)))

def abcs_damp(h, counts, offsets, y, n_img, H, W, B, iters, damping, denoiser, lam, cnn_weights, probe, x_out,
              sigma_trace=None, alpha_trace=None, stream=None) -> None:
    """D-AMP (damping 1) / DAMP-D: IDA with the Onsager coefficient from the
    Monte-Carlo divergence of the denoiser with the given probe."""
    _check(lib.abcs_damp(h, _ptr(counts), _ptr(offsets), _ptr(y), n_img, H, W, B, iters, damping, denoiser, lam,
                         _ptr(cnn_weights), _ptr(probe), _ptr(x_out), _ptr(sigma_trace), _ptr(alpha_trace),
                         _stream(stream)))


def abcs_thi(h, coeffs, n_img, H, W, B, M, adaptive, thi_counts, rho=None, masked=None, stream=None) -> None:
    """THI: per image the M coefficients of largest magnitude (coeffs: every
    coefficient, zigzag order per block); thi_counts per block, rho against
    `adaptive` counts (or None), masked coefficients (or None)."""
    _check(lib.abcs_thi(h, _ptr(coeffs), n_img, H, W, B, M, _ptr(adaptive), _ptr(thi_counts), _ptr(rho),
                        _ptr(masked), _stream(stream)))


def abcs_psnr_ssim(h, x, ref, n_img, H, W, ref_pitch, ref_stride, psnr, ssim, stream=None) -> None:
    """psnr, ssim [n_img] float64 device tensors <- the quality of x against ref."""
    _check(lib.abcs_psnr_ssim(h, _ptr(x), _ptr(ref), n_img, H, W, ref_pitch, ref_stride, _ptr(psnr), _ptr(ssim),
                              _stream(stream)))


def abcs_set_ida_precision(h, precision) -> None:
    """Transform precision of the IDA linear step on this handle (FP32 or a
    tensor-core precision, used for B = 16)."""
    _check(lib.abcs_set_ida_precision(h, precision))


def abcs_sync_status(h, stream=None) -> int:
    """Waits for the stream; returns the device status bits (0 = clean)."""
    bits = C.c_uint32(0)
    st = lib.abcs_sync_status(h, _stream(stream), C.byref(bits))
    if st not in (0, 8):
        _check(st)
    return bits.value
