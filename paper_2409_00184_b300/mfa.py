"""Python binding of libmfa.so (the C ABI declared in include/mfa.h): argument marshalling only.

Every function here forwards device pointers (torch tensors on the CUDA device), sizes and a
CUDA stream to the library; all arithmetic runs in the library's kernels. Importing this module
fails loudly if the compiled library is missing: there is no CPU or framework fallback.
"""

import ctypes
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmfa.so")

OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_CAPACITY, ERR_DEVICE, ERR_IO = -1, -2, -3, -4, -5, -6, -7
DEV_BAD_DESC, DEV_BAD_KNOTS, DEV_BAD_RANGE, DEV_BAD_LIST, DEV_TIMEOUT, DEV_NOT_SPD = 1, 2, 4, 8, 16, 32
PREC_FP32, PREC_BF16, PREC_FP16, PREC_SPLIT_BF16 = 0, 1, 2, 3
DECODE_VALUE_ONLY, DECODE_LIST_SLOTS, DECODE_CUBES, DECODE_APRON = 1, 2, 4, 8
RAYCAST_CUBES, RAYCAST_APRON, RAYCAST_COUNT_SECTORS = 1, 2, 4
STAT_RAY_SAMPLES, STAT_RAY_SECTORS, NUM_STATS = 0, 1, 2
LOD_SHARED_BOUNDARY = 1
MAX_DEGREE, MAX_NCP, MAX_NSAMP = 3, 32, 64


class BlockDesc(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32 * 3), ("ncp", ctypes.c_int32 * 3), ("nsamp", ctypes.c_int32 * 3),
                ("slot", ctypes.c_int32), ("knot_off", ctypes.c_int64 * 3), ("cp_off", ctypes.c_int64)]


class Bounds(ctypes.Structure):
    _fields_ = [("max_degree", ctypes.c_int32), ("max_ncp", ctypes.c_int32), ("max_nsamp", ctypes.c_int32)]


class DecodeTiling(ctypes.Structure):
    _fields_ = [("ks", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32)]


class View(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fov_y_deg", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("step_voxels", ctypes.c_float), ("opacity_max", ctypes.c_float), ("ka", ctypes.c_float),
                ("kd", ctypes.c_float), ("ks", ctypes.c_float), ("shininess", ctypes.c_float),
                ("vmin", ctypes.c_float), ("vmax", ctypes.c_float)]


class FrameDesc(ctypes.Structure):
    _fields_ = [("d_desc", ctypes.c_void_p), ("nblocks", ctypes.c_int32), ("d_list", ctypes.c_void_p),
                ("list_capacity", ctypes.c_int32), ("d_count", ctypes.c_void_p), ("d_knots", ctypes.c_void_p),
                ("knots_len", ctypes.c_int64), ("d_cps", ctypes.c_void_p), ("cps_len", ctypes.c_int64),
                ("d_cache", ctypes.c_void_p), ("slot_stride_voxels", ctypes.c_int64), ("bounds", Bounds),
                ("flags", ctypes.c_uint32), ("d_brick_table", ctypes.c_void_p), ("brick_dims", ctypes.c_int32 * 3),
                ("brick_n", ctypes.c_int32), ("view", ctypes.c_void_p), ("d_tf", ctypes.c_void_p),
                ("tf_n", ctypes.c_int32), ("d_image", ctypes.c_void_p), ("precision", ctypes.c_int32)]


FRAME_SORT_BY_COST, FRAME_RAYCAST, FRAME_CUBES, FRAME_APRON = 1, 2, 4, 8

DESC_DTYPE = np.dtype({"names": ["degree", "ncp", "nsamp", "slot", "knot_off", "cp_off"],
                       "formats": [("<i4", 3), ("<i4", 3), ("<i4", 3), "<i4", ("<i8", 3), "<i8"],
                       "offsets": [0, 12, 24, 36, 40, 64], "itemsize": 72})
assert ctypes.sizeof(BlockDesc) == DESC_DTYPE.itemsize == 72

SYMBOLS = ["mfa_abi_struct_sizes", "mfa_ctx_create", "mfa_ctx_destroy", "mfa_status_string", "mfa_ctx_device_status",
           "mfa_ctx_launch_count", "mfa_model_bytes", "mfa_decode_blocks", "mfa_basis_tables",
           "mfa_adjoint_blocks", "mfa_encode_plan_create", "mfa_encode_plan_destroy", "mfa_encode_blocks",
           "mfa_raycast", "mfa_ctx_set_decode_tiling", "mfa_ctx_get_decode_tiling", "mfa_encode_blocks_noalloc",
           "mfa_frame_graph_create", "mfa_frame_graph_launch", "mfa_frame_graph_destroy",
           "mfa_ctx_read_stats", "mfa_select_ncp", "mfa_selftest_wait_timeout", "mfa_lod_gather",
           "mfa_raycast_direct", "mfa_decode_compare_blocks", "mfa_store_write", "mfa_cache_create", "mfa_cache_destroy", "mfa_cache_info",
           "mfa_cache_lookup", "mfa_cache_upload", "mfa_cache_prefetch_start", "mfa_cache_prefetch_stop",
           "mfa_raycast_ex", "mfa_fill_aprons", "mfa_lod_gather_ex", "mfa_lod_select", "mfa_raycast_lod",
           "mfa_encode_blocks_ex", "mfa_copy_to_device", "mfa_copy_to_host"]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libmfa.so not found at {_LIB_PATH}: build it with "
                          "`python -m paper_2409_00184_b300.build` (no fallback path exists)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "mfa_ctx_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int]),
        "mfa_ctx_destroy": (None, [P]),
        "mfa_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "mfa_abi_struct_sizes": (ctypes.c_int, [P, I32]),
        "mfa_ctx_device_status": (ctypes.c_int, [P, ctypes.POINTER(U32), ctypes.c_int, P]),
        "mfa_ctx_launch_count": (I64, [P]),
        "mfa_ctx_set_decode_tiling": (ctypes.c_int, [P, ctypes.POINTER(Bounds), ctypes.POINTER(DecodeTiling)]),
        "mfa_ctx_get_decode_tiling": (ctypes.c_int, [P, ctypes.POINTER(Bounds), ctypes.POINTER(DecodeTiling)]),
        "mfa_model_bytes": (I64, [I32, I32]),
        "mfa_copy_to_device": (ctypes.c_int, [P, P, I64, P]),
        "mfa_copy_to_host": (ctypes.c_int, [P, P, I64, P]),
        "mfa_decode_blocks": (ctypes.c_int, [P, P, I32, P, I32, P, P, I64, P, I64, P, I64, I64,
                                             ctypes.POINTER(Bounds), I32, U32, P]),
        "mfa_basis_tables": (ctypes.c_int, [P, P, P, I64, P, P, P]),
        "mfa_adjoint_blocks": (ctypes.c_int, [P, P, I32, P, I64, P, I64, I64, P, P, I64,
                                              ctypes.POINTER(Bounds), I32, P]),
        "mfa_encode_plan_create": (ctypes.c_int, [P, ctypes.POINTER(P), P, I32, P, I64, I64]),
        "mfa_encode_plan_destroy": (None, [P]),
        "mfa_encode_blocks": (ctypes.c_int, [P, P, P, I64, I64, P, P, P]),
        "mfa_encode_blocks_ex": (ctypes.c_int, [P, P, P, I64, I64, P, P, I32, P]),
        "mfa_encode_blocks_noalloc": (ctypes.c_int, [P, I32, P, I64, P, I64, I64, P, I64, P, P]),
        "mfa_select_ncp": (ctypes.c_int, [P, P, I32, P, I64, ctypes.c_double, P, P]),
        "mfa_selftest_wait_timeout": (ctypes.c_int, [P, I32, P]),
        "mfa_lod_gather": (ctypes.c_int, [P, P, ctypes.POINTER(I32), I32, I32, P, I32, P, I64, P]),
        "mfa_lod_gather_ex": (ctypes.c_int, [P, P, ctypes.POINTER(I32), I32, I32, P, I32, P, I64, U32, P]),
        "mfa_lod_select": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_float * 3), I32, I32, I32, P, P, P]),
        "mfa_raycast_lod": (ctypes.c_int, [P, P, I32, P, I64, P, I64, ctypes.POINTER(Bounds), P, I32, I32, I32,
                                           ctypes.POINTER(View), P, I32, P, P]),
        "mfa_raycast_direct": (ctypes.c_int, [P, P, I32, P, I64, P, I64, ctypes.POINTER(Bounds), P,
                                              ctypes.POINTER(I32), I32, P, P, I32, P, P]),
        "mfa_store_write": (ctypes.c_int, [ctypes.c_char_p, P, I32, P, I64, P, I64]),
        "mfa_decode_compare_blocks": (ctypes.c_int, [P, P, I32, P, I32, P, P, I64, P, I64, P, I64, I64,
                                                     ctypes.POINTER(Bounds), U32, P, I64, P, P, P]),
        "mfa_cache_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_char_p, I32, I32]),
        "mfa_cache_destroy": (None, [P]),
        "mfa_cache_info": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "mfa_cache_lookup": (ctypes.c_int, [P, P, I32, P]),
        "mfa_cache_upload": (ctypes.c_int, [P, P, I32, I32, P, P, I64, P, I64, P, ctypes.POINTER(Bounds), P]),
        "mfa_cache_prefetch_start": (ctypes.c_int, [P, P, I32]),
        "mfa_cache_prefetch_stop": (ctypes.c_int, [P, P]),
        "mfa_frame_graph_create": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(FrameDesc)]),
        "mfa_frame_graph_launch": (ctypes.c_int, [P, P]),
        "mfa_frame_graph_destroy": (None, [P]),
        "mfa_ctx_read_stats": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int, P]),
        "mfa_raycast": (ctypes.c_int, [P, P, I64, I64, P, ctypes.POINTER(ctypes.c_int32 * 3), I32,
                                       ctypes.POINTER(View), P, I32, P, P]),
        "mfa_raycast_ex": (ctypes.c_int, [P, P, I64, I64, P, ctypes.POINTER(ctypes.c_int32 * 3), I32,
                                          ctypes.POINTER(View), P, I32, P, ctypes.c_uint32, P]),
        "mfa_fill_aprons": (ctypes.c_int, [P, P, I64, I64, P, ctypes.POINTER(ctypes.c_int32 * 3), I32, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def abi_struct_sizes():
    """mfa_abi_struct_sizes: the C sizes of mfa_block_desc, mfa_bounds, mfa_decode_tiling, mfa_view and
    mfa_frame_desc, in that order (host only)."""
    n = lib.mfa_abi_struct_sizes(None, 0)
    out = (ctypes.c_int32 * n)()
    lib.mfa_abi_struct_sizes(ctypes.cast(out, ctypes.c_void_p), n)
    return list(out)


class MfaError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {lib.mfa_status_string(code).decode()} ({code})")
        self.code = code


def _check(code, what):
    if code != OK:
        raise MfaError(code, what)


F32, F64, I32, U8 = torch.float32, torch.float64, torch.int32, torch.uint8


def _ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None stays None). With dtype, the tensor must hold that
    element type: the library reads and writes it with that width, and the element counts checked against
    the call's extents assume it."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected a {dtype} tensor, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _tf(tf):
    """Pointer and entry count of a transfer function: a float32 CUDA tensor of shape (n, 4) (RGBA)."""
    if tf.dim() != 2 or tf.shape[1] != 4:
        raise ValueError("tf: float32 tensor of shape (n, 4)")
    return _ptr(tf, F32), tf.shape[0]


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host_ptr(t):
    if t.is_cuda:
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, n, what):
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call touches {n}")


def apron_pitch(n):
    """Row pitch (voxels) of a brick with n voxels per row in the DECODE_APRON layout: n + 1 rounded up to even."""
    return (n + 2) & ~1


def apron_voxels(n):
    """Smallest slot stride (voxels) of an n^3 brick in the DECODE_APRON layout."""
    return apron_pitch(n) * (n + 1) ** 2


def model_bytes(ncp, degree):
    """Eq. 2 model size in bytes."""
    return int(lib.mfa_model_bytes(ncp, degree))


def copy_to_device(dst, src, stream=None):
    """mfa_copy_to_device: the bytes of host tensor src (page-locked for an asynchronous copy) into CUDA
    tensor dst."""
    if dst.numel() * dst.element_size() < src.numel() * src.element_size():
        raise ValueError("destination smaller than source")
    _check(lib.mfa_copy_to_device(_ptr(dst), _host_ptr(src), src.numel() * src.element_size(), _stream(stream)),
           "mfa_copy_to_device")


def copy_to_host(dst, src, stream=None):
    """mfa_copy_to_host: the bytes of CUDA tensor src into host tensor dst (page-locked for an asynchronous
    copy)."""
    if dst.numel() * dst.element_size() < src.numel() * src.element_size():
        raise ValueError("destination smaller than source")
    _check(lib.mfa_copy_to_host(_host_ptr(dst), _ptr(src), src.numel() * src.element_size(), _stream(stream)),
           "mfa_copy_to_host")


class Context:
    """An mfa_ctx on one CUDA device."""

    def __init__(self, device=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        torch.cuda.init()
        self.device = dev
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _check(lib.mfa_ctx_create(ctypes.byref(h), dev.index), "mfa_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib.mfa_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self, clear=True, stream=None):
        st = ctypes.c_uint32()
        _check(lib.mfa_ctx_device_status(self.handle, ctypes.byref(st), int(clear), _stream(stream)),
               "mfa_ctx_device_status")
        return st.value

    def launch_count(self):
        return int(lib.mfa_ctx_launch_count(self.handle))

    def selftest_wait_timeout(self, polls=1000, stream=None):
        """mfa_selftest_wait_timeout: a bounded wait on a barrier nothing arrives on (sets MFA_DEV_TIMEOUT)."""
        _check(lib.mfa_selftest_wait_timeout(self.handle, int(polls), _stream(stream)), "mfa_selftest_wait_timeout")

    def ray_samples(self, reset=True, stream=None):
        """Samples marched by mfa_raycast since the last reset (synchronises the stream; resets every
        statistic)."""
        return self.stats(reset, stream)[0]

    def stats(self, reset=True, stream=None):
        """Every MFA_STAT_* counter (ray samples, ray-cast sectors) since the last reset (synchronises)."""
        v = (ctypes.c_uint64 * NUM_STATS)()
        _check(lib.mfa_ctx_read_stats(self.handle, v, NUM_STATS, int(reset), _stream(stream)), "mfa_ctx_read_stats")
        return [int(x) for x in v]

    def set_decode_tiling(self, bounds, ks=0, ctas_per_sm=0):
        _check(lib.mfa_ctx_set_decode_tiling(self.handle, ctypes.byref(bounds),
                                             ctypes.byref(DecodeTiling(ks, ctas_per_sm))), "mfa_ctx_set_decode_tiling")

    def get_decode_tiling(self, bounds):
        t = DecodeTiling()
        rc = lib.mfa_ctx_get_decode_tiling(self.handle, ctypes.byref(bounds), ctypes.byref(t))
        return (t.ks, t.ctas_per_sm) if rc == OK else None


def pack_descriptors(bs):
    """numpy structured array (72-byte records) of a synth.BlockSet's descriptors."""
    d = np.zeros(len(bs), dtype=DESC_DTYPE)
    d["degree"], d["ncp"], d["nsamp"] = bs.degree, bs.ncp, bs.nsamp
    d["slot"], d["knot_off"], d["cp_off"] = bs.slot, bs.knot_off, bs.cp_off
    return d


def bounds_of(bs):
    return Bounds(int(np.max(bs.degree)), int(np.max(bs.ncp)), int(np.max(bs.nsamp)))


class DeviceBlocks:
    """A batch of micro-models resident on the device: descriptors, knots, control points."""

    def __init__(self, bs, device="cuda", cps=None):
        self.n = len(bs)
        self.host_desc = pack_descriptors(bs)
        self.desc = torch.from_numpy(self.host_desc.view(np.uint8).copy()).to(device)
        self.host_knots = np.ascontiguousarray(bs.knots, dtype=np.float32)
        self.knots = torch.from_numpy(self.host_knots).to(device)
        self.cps = cps if cps is not None else torch.from_numpy(np.ascontiguousarray(bs.cps, np.float32)).to(device)
        self.bounds = bounds_of(bs)
        self.slot_voxels = int(np.max(np.prod(bs.nsamp.astype(np.int64), axis=1)))
        self.nslots = int(np.max(bs.slot)) + 1 if self.n else 0
        self.cps_len = int(np.sum(np.prod(bs.ncp.astype(np.int64), axis=1)))


def decode_blocks(ctx, blocks, cache, slot_stride, nslots, precision=PREC_FP32, flags=0, cps=None,
                  list_=None, count=None, bounds=None, stream=None):
    """mfa_decode_blocks on a DeviceBlocks batch; cache: float32 CUDA tensor."""
    cps = blocks.cps if cps is None else cps
    if list_ is not None and list_.numel() == 0:
        return  # an empty list selects nothing (a NULL list would mean every block)
    width = 1 if flags & DECODE_VALUE_ONLY else 4
    _need(cache, nslots * slot_stride * width, "cache")
    _need(cps, blocks.cps_len, "cps")
    _check(lib.mfa_decode_blocks(ctx.handle, _ptr(blocks.desc), blocks.n,
                                 _ptr(list_, I32), 0 if list_ is None else list_.numel(), _ptr(count, I32),
                                 _ptr(blocks.knots), blocks.knots.numel(), _ptr(cps, F32), cps.numel(),
                                 _ptr(cache, F32), slot_stride, nslots, ctypes.byref(bounds or blocks.bounds),
                                 precision, flags, _stream(stream)), "mfa_decode_blocks")


def decode_compare_blocks(ctx, blocks, cache, slot_stride, nslots, data, data_stride, residual=None, rmse=None,
                          flags=0, cps=None, list_=None, count=None, bounds=None, stream=None):
    """mfa_decode_compare_blocks: the FP32 decode of decode_blocks and, in the same pass, r = f - D against the
    sample grids `data` (slot-addressed, data_stride floats per slot): residual (optional, same addressing)
    and the RMSE per selected item (optional float64 tensor)."""
    cps = blocks.cps if cps is None else cps
    if list_ is not None and list_.numel() == 0:
        return
    width = 1 if flags & DECODE_VALUE_ONLY else 4
    _need(cache, nslots * slot_stride * width, "cache")
    _need(cps, blocks.cps_len, "cps")
    _need(data, nslots * data_stride, "data")
    if residual is not None:
        _need(residual, nslots * data_stride, "residual")
    if rmse is not None:
        if rmse.dtype != torch.float64:
            raise ValueError("rmse: float64 tensor")
        _need(rmse, list_.numel() if list_ is not None else blocks.n, "rmse")
    _check(lib.mfa_decode_compare_blocks(ctx.handle, _ptr(blocks.desc), blocks.n, _ptr(list_, I32),
                                         0 if list_ is None else list_.numel(), _ptr(count, I32), _ptr(blocks.knots),
                                         blocks.knots.numel(), _ptr(cps, F32), cps.numel(), _ptr(cache, F32),
                                         slot_stride, nslots, ctypes.byref(bounds or blocks.bounds), flags,
                                         _ptr(data, F32), data_stride, _ptr(residual, F32), _ptr(rmse, F64),
                                         _stream(stream)), "mfa_decode_compare_blocks")


def basis_tables(ctx, desc_one, knots, stream=None):
    """mfa_basis_tables for one descriptor (uint8 CUDA tensor of 72 bytes): (span (3, 64), basis (3, 64, 2, 4))."""
    span = torch.zeros(3 * MAX_NSAMP, dtype=torch.int32, device=knots.device)
    basis = torch.zeros(3 * MAX_NSAMP * 2 * 4, dtype=torch.float32, device=knots.device)
    _check(lib.mfa_basis_tables(ctx.handle, _ptr(desc_one, U8), _ptr(knots, F32), knots.numel(), _ptr(span),
                                _ptr(basis),
                                _stream(stream)), "mfa_basis_tables")
    return span.view(3, MAX_NSAMP), basis.view(3, MAX_NSAMP, 2, 4)


def adjoint_blocks(ctx, blocks, residual, slot_stride, nslots, grad, cps=None, precision=PREC_FP32,
                   bounds=None, stream=None):
    """mfa_adjoint_blocks: grad <- N^T residual per block (or N^T (decode(cps) - residual) with cps)."""
    _need(residual, nslots * slot_stride, "residual")
    _need(grad, blocks.cps_len, "grad")
    if cps is not None:
        _need(cps, blocks.cps_len, "cps")
    _check(lib.mfa_adjoint_blocks(ctx.handle, _ptr(blocks.desc), blocks.n, _ptr(blocks.knots), blocks.knots.numel(),
                                  _ptr(residual, F32), slot_stride, nslots, _ptr(cps, F32), _ptr(grad, F32),
                                  grad.numel(),
                                  ctypes.byref(bounds or blocks.bounds), precision, _stream(stream)),
           "mfa_adjoint_blocks")


class EncodePlan:
    """mfa_encode_plan for a DeviceBlocks batch (validated and grouped into axis classes on the host)."""

    def __init__(self, ctx, blocks):
        self.ctx = ctx
        h = ctypes.c_void_p()
        desc = np.ascontiguousarray(blocks.host_desc)
        _check(lib.mfa_encode_plan_create(ctx.handle, ctypes.byref(h), desc.ctypes.data_as(ctypes.c_void_p),
                                          blocks.n, blocks.host_knots.ctypes.data_as(ctypes.c_void_p),
                                          blocks.host_knots.size, blocks.cps_len), "mfa_encode_plan_create")
        self.handle = h
        self.cps_len, self.nblocks = blocks.cps_len, blocks.n

    def close(self):
        if self.handle:
            lib.mfa_encode_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode_blocks(ctx, plan, data, slot_stride, nslots, cps_out, rmse=None, stream=None, precision=PREC_FP32):
    """mfa_encode_blocks (mfa_encode_blocks_ex for another precision): least-squares control points (and FP64
    RMSE per block, FP32 only) from sample grids."""
    _need(data, nslots * slot_stride, "data")
    _need(cps_out, plan.cps_len, "cps_out")
    if rmse is not None:
        _need(rmse, plan.nblocks, "rmse")
    if precision == PREC_FP32:
        _check(lib.mfa_encode_blocks(ctx.handle, plan.handle, _ptr(data, F32), slot_stride, nslots,
                                     _ptr(cps_out, F32), _ptr(rmse, F64), _stream(stream)), "mfa_encode_blocks")
    else:
        _check(lib.mfa_encode_blocks_ex(ctx.handle, plan.handle, _ptr(data, F32), slot_stride, nslots,
                                        _ptr(cps_out, F32), _ptr(rmse, F64), precision, _stream(stream)),
               "mfa_encode_blocks_ex")


def encode_blocks_noalloc(blocks, data, slot_stride, nslots, cps_out, rmse=None, stream=None):
    """mfa_encode_blocks_noalloc: the least-squares fit with the library's fixed device scratch (no context,
    no plan, no device allocation); synchronises the stream before returning."""
    _need(data, nslots * slot_stride, "data")
    _need(cps_out, blocks.cps_len, "cps_out")
    if rmse is not None:
        _need(rmse, blocks.n, "rmse")
    desc = np.ascontiguousarray(blocks.host_desc)
    rc = lib.mfa_encode_blocks_noalloc(desc.ctypes.data_as(ctypes.c_void_p), blocks.n,
                                       blocks.host_knots.ctypes.data_as(ctypes.c_void_p), blocks.host_knots.size,
                                       _ptr(data, F32), slot_stride, nslots, _ptr(cps_out, F32), blocks.cps_len,
                                       _ptr(rmse, F64),
                                       _stream(stream))
    if rc == ERR_CAPACITY:
        raise MfaError(rc, "mfa_encode_blocks_noalloc: the batch's tables exceed the fixed 2 MiB scratch")
    _check(rc, "mfa_encode_blocks_noalloc")


def select_ncp(ctx, errors, ncps, bound, out=None, stream=None):
    """mfa_select_ncp (Eq. 4): errors is a float64 CUDA tensor (len(ncps), nblocks), candidate-major; returns
    (or fills) an int32 CUDA tensor with, per block, the smallest candidate NCP whose error is below `bound`,
    or -1."""
    ncand = len(ncps)
    if errors.dtype != torch.float64 or errors.dim() != 2 or errors.shape[0] != ncand:
        raise ValueError("errors: float64 tensor of shape (len(ncps), nblocks)")
    nb = errors.shape[1]
    if out is None:
        out = torch.empty(nb, dtype=torch.int32, device=errors.device)
    _need(out, nb, "out")
    h = (ctypes.c_int32 * ncand)(*[int(c) for c in ncps])
    _check(lib.mfa_select_ncp(ctx.handle, _ptr(errors, F64), ncand, h, nb, float(bound), _ptr(out, I32),
                              _stream(stream)),
           "mfa_select_ncp")
    return out


def lod_gather(ctx, field, n, stride, ids=None, nblocks=None, out=None, stream=None, shared=False):
    """mfa_lod_gather (mfa_lod_gather_ex with MFA_LOD_SHARED_BOUNDARY when shared): the n^3 micro-blocks of
    one level of detail (every stride-th sample of blocks of n*stride samples per axis, or of (n-1)*stride
    intervals sharing their boundary samples) of a float32 CUDA field of shape (Nz, Ny, Nx). ids: int32
    CUDA tensor of block ids (None = the first nblocks, default all). Returns a float32 tensor (len, n^3)."""
    if field.dim() != 3:
        raise ValueError("field: (Nz, Ny, Nx) tensor")
    Nz, Ny, Nx = field.shape
    if shared:
        span = (n - 1) * stride
        total = ((Nx - 1) // span) * ((Ny - 1) // span) * ((Nz - 1) // span)
    else:
        span = n * stride
        total = (Nx // span) * (Ny // span) * (Nz // span)
    count = ids.numel() if ids is not None else (total if nblocks is None else nblocks)
    if out is None:
        out = torch.empty((count, n ** 3), dtype=torch.float32, device=field.device)
    _need(out, count * n ** 3, "out")
    dims = (ctypes.c_int32 * 3)(Nx, Ny, Nz)
    if count == 0:
        return out
    _check(lib.mfa_lod_gather_ex(ctx.handle, _ptr(field, F32), dims, n, stride, _ptr(ids, I32), count,
                                 _ptr(out, F32), n ** 3,
                                 LOD_SHARED_BOUNDARY if shared else 0, _stream(stream)), "mfa_lod_gather_ex")
    return out


def lod_select(ctx, eye, fine_blocks, n, levels, ranges=(0.8, 1.6, 2.4), table=None, stream=None):
    """mfa_lod_select: int32 CUDA tensor (B0, B0, B0) [z][y][x] of the global id of the block that covers every
    finest block for a point of view (levels of detail by distance, ranges[l-1] for level l >= 1)."""
    if table is None:
        table = torch.empty((fine_blocks,) * 3, dtype=torch.int32, device="cuda")
    _need(table, fine_blocks ** 3, "table")
    e = (ctypes.c_float * 3)(*[float(x) for x in eye])
    r = (ctypes.c_float * max(1, len(ranges)))(*[float(x) for x in ranges])
    _check(lib.mfa_lod_select(ctx.handle, ctypes.byref(e), fine_blocks, n, levels, r if levels > 1 else None,
                              _ptr(table, I32), _stream(stream)), "mfa_lod_select")
    return table


def raycast_lod(ctx, blocks, table, fine_blocks, n, levels, view, tf, image, cps=None, stream=None):
    """mfa_raycast_lod: Algorithm 4 with per-sample queries of the models `table` (from lod_select) picks in a
    DeviceBlocks batch holding every level's blocks by global id; image a float32 (H, W, 4) CUDA tensor."""
    cps = blocks.cps if cps is None else cps
    _need(image, int(view["width"]) * int(view["height"]) * 4, "image")
    _need(table, fine_blocks ** 3, "table")
    v = make_view(view)
    tfp, tfn = _tf(tf)
    _check(lib.mfa_raycast_lod(ctx.handle, _ptr(blocks.desc), blocks.n, _ptr(blocks.knots), blocks.knots.numel(),
                               _ptr(cps, F32), cps.numel(), ctypes.byref(blocks.bounds), _ptr(table, I32),
                               fine_blocks, n, levels, ctypes.byref(v), tfp, tfn, _ptr(image, F32), _stream(stream)),
           "mfa_raycast_lod")


def store_write(path, bs):
    """mfa_store_write: every block of a host batch (synth.BlockSet-like arrays) into a store file."""
    desc = pack_descriptors(bs)
    knots = np.ascontiguousarray(bs.knots, dtype=np.float32)
    cps = np.ascontiguousarray(bs.cps, dtype=np.float32)
    _check(lib.mfa_store_write(str(path).encode(), desc.ctypes.data_as(ctypes.c_void_p), len(desc),
                               knots.ctypes.data_as(ctypes.c_void_p), knots.size,
                               cps.ctypes.data_as(ctypes.c_void_p), cps.size), "mfa_store_write")


def _host_ids(ids):
    a = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.c_void_p)


class DeviceBatch:
    """Device buffers for up to `capacity` uploaded models of at most max_ncp^3 control points (the
    attributes decode_blocks and raycast_direct read: desc, knots, cps, n, bounds)."""

    def __init__(self, capacity, max_ncp, max_degree, device="cuda"):
        self.desc = torch.zeros(capacity * 72, dtype=torch.uint8, device=device)
        self.knots = torch.zeros(capacity * 3 * (max_ncp + max_degree + 1), dtype=torch.float32, device=device)
        self.cps = torch.zeros(capacity * max_ncp ** 3, dtype=torch.float32, device=device)
        self.n, self.bounds, self.cps_len = 0, Bounds(1, 2, 2), 0


class ModelCache:
    """mfa_model_cache: LRU cache of a store's micro-models in host memory (Algorithms 2 and 3)."""

    def __init__(self, path, capacity, pinned=True):
        h = ctypes.c_void_p()
        _check(lib.mfa_cache_create(ctypes.byref(h), str(path).encode(), int(capacity), int(bool(pinned))),
               "mfa_cache_create")
        self.handle, self.capacity = h, capacity

    def info(self):
        c, mc, md = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.mfa_cache_info(self.handle, ctypes.byref(c), ctypes.byref(mc), ctypes.byref(md)), "mfa_cache_info")
        return c.value, mc.value, md.value

    def lookup(self, ids):
        a, p = _host_ids(ids)
        st = (ctypes.c_int64 * 4)()
        _check(lib.mfa_cache_lookup(self.handle, p, a.size, st), "mfa_cache_lookup")
        return {"hits": st[0], "misses": st[1], "bytes": st[2], "ns": st[3]}

    def upload(self, ids, nsamp, batch, stream=None):
        a, p = _host_ids(ids)
        lens = (ctypes.c_int64 * 2)()
        _check(lib.mfa_cache_upload(self.handle, p, a.size, nsamp, _ptr(batch.desc), _ptr(batch.knots),
                                    batch.knots.numel(), _ptr(batch.cps), batch.cps.numel(), lens,
                                    ctypes.byref(batch.bounds), _stream(stream)), "mfa_cache_upload")
        batch.n, batch.cps_len = a.size, lens[1]
        return batch

    def prefetch_start(self, ids):
        a, p = _host_ids(ids)
        self._pf = a  # the thread copies the list; kept only for clarity
        _check(lib.mfa_cache_prefetch_start(self.handle, p, a.size), "mfa_cache_prefetch_start")

    def prefetch_stop(self):
        st = (ctypes.c_int64 * 2)()
        _check(lib.mfa_cache_prefetch_stop(self.handle, st), "mfa_cache_prefetch_stop")
        return {"loaded": st[0], "bytes": st[1]}

    def close(self):
        if self.handle:
            lib.mfa_cache_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_view(v):
    return View((ctypes.c_float * 3)(*v["eye"]), (ctypes.c_float * 3)(*v["target"]),
                (ctypes.c_float * 3)(*v["up"]), v["fov_y_deg"], int(v["width"]), int(v["height"]),
                v.get("step_voxels", 1.0), v["opacity_max"], v["ka"], v["kd"], v["ks"], v["shininess"],
                v["vmin"], v["vmax"])


def raycast_direct(ctx, blocks, table, brick_n, view, tf, image, cps=None, stream=None):
    """mfa_raycast_direct: per-sample queries of the micro-models of a DeviceBlocks batch; table is an int32
    (Bz, By, Bx) CUDA tensor of block indices (-1 = absent), image a float32 (H, W, 4) CUDA tensor."""
    cps = blocks.cps if cps is None else cps
    Bz, By, Bx = table.shape
    _need(image, int(view["width"]) * int(view["height"]) * 4, "image")
    v = make_view(view)
    dims = (ctypes.c_int32 * 3)(Bx, By, Bz)
    tfp, tfn = _tf(tf)
    _check(lib.mfa_raycast_direct(ctx.handle, _ptr(blocks.desc), blocks.n, _ptr(blocks.knots), blocks.knots.numel(),
                                  _ptr(cps, F32), cps.numel(), ctypes.byref(blocks.bounds), _ptr(table, I32), dims,
                                  brick_n, ctypes.byref(v), tfp, tfn, _ptr(image, F32), _stream(stream)),
           "mfa_raycast_direct")


def raycast(ctx, cache, slot_stride, nslots, table, brick_n, view, tf, image, stream=None, cubes=False,
            apron=False, count_sectors=False):
    """mfa_raycast (mfa_raycast_ex with MFA_RAYCAST_CUBES, MFA_RAYCAST_APRON or MFA_RAYCAST_COUNT_SECTORS):
    table is an int32 (Bz, By, Bx) CUDA tensor; image a float32 (H, W, 4) CUDA tensor."""
    Bz, By, Bx = table.shape
    _need(image, int(view["width"]) * int(view["height"]) * 4, "image")
    _need(cache, nslots * slot_stride * 4, "cache")
    dims = (ctypes.c_int32 * 3)(Bx, By, Bz)
    vw = make_view(view)
    tfp, tfn = _tf(tf)
    if cubes or apron or count_sectors:
        flags = ((RAYCAST_CUBES if cubes else 0) | (RAYCAST_APRON if apron else 0) |
                 (RAYCAST_COUNT_SECTORS if count_sectors else 0))
        _check(lib.mfa_raycast_ex(ctx.handle, _ptr(cache, F32), slot_stride, nslots, _ptr(table, I32),
                                  ctypes.byref(dims), brick_n, ctypes.byref(vw), tfp, tfn, _ptr(image, F32), flags,
                                  _stream(stream)), "mfa_raycast_ex")
    else:
        _check(lib.mfa_raycast(ctx.handle, _ptr(cache, F32), slot_stride, nslots, _ptr(table, I32),
                               ctypes.byref(dims), brick_n, ctypes.byref(vw), tfp, tfn, _ptr(image, F32),
                               _stream(stream)),
               "mfa_raycast")


def fill_aprons(ctx, cache, slot_stride, nslots, table, brick_n, stream=None):
    """mfa_fill_aprons: the apron planes of every brick of `table` (int32 (Bz, By, Bx) CUDA tensor) in a cache
    decoded with DECODE_APRON (slot_stride >= apron_voxels(brick_n) voxels of 4 floats)."""
    Bz, By, Bx = table.shape
    _need(cache, nslots * slot_stride * 4, "cache")
    dims = (ctypes.c_int32 * 3)(Bx, By, Bz)
    _check(lib.mfa_fill_aprons(ctx.handle, _ptr(cache, F32), slot_stride, nslots, _ptr(table, I32), ctypes.byref(dims),
                               brick_n, _stream(stream)), "mfa_fill_aprons")


class FrameGraph:
    """mfa_frame_graph: one frame (cost ordering, decode of the visible list, brick table, ray cast)
    captured as a CUDA graph. Write the visible ids into `list_buf` and their number into `count_buf`
    (device int32 tensors) before each launch()."""

    def __init__(self, ctx, blocks, list_buf, count_buf, cache, slot_stride, sort=True,
                 table=None, brick_dims=None, brick_n=0, view=None, tf=None, image=None, cubes=False,
                 apron=False, precision=PREC_FP32):
        self.ctx = ctx
        self._keep = [blocks, list_buf, count_buf, cache, table, tf, image]
        cap = list_buf.numel()
        _need(cache, cap * slot_stride * 4, "cache")
        flags = (FRAME_SORT_BY_COST if sort else 0) | (FRAME_CUBES if cubes else 0) | (FRAME_APRON if apron else 0)
        self._view = None
        fd = FrameDesc()
        fd.d_desc, fd.nblocks = _ptr(blocks.desc), blocks.n
        fd.d_list, fd.list_capacity, fd.d_count = _ptr(list_buf, I32), cap, _ptr(count_buf, I32)
        fd.d_knots, fd.knots_len = _ptr(blocks.knots), blocks.knots.numel()
        fd.d_cps, fd.cps_len = _ptr(blocks.cps, F32), blocks.cps.numel()
        fd.d_cache, fd.slot_stride_voxels = _ptr(cache, F32), slot_stride
        fd.bounds = blocks.bounds
        fd.precision = precision
        if view is not None:
            flags |= FRAME_RAYCAST
            _need(table, blocks.n, "table")
            _need(image, int(view["width"]) * int(view["height"]) * 4, "image")
            self._view = make_view(view)
            fd.d_brick_table = _ptr(table, I32)
            fd.brick_dims = (ctypes.c_int32 * 3)(*brick_dims)
            fd.brick_n = brick_n
            fd.view = ctypes.cast(ctypes.pointer(self._view), ctypes.c_void_p)
            fd.d_tf, fd.tf_n = _tf(tf)
            fd.d_image = _ptr(image, F32)
        fd.flags = flags
        h = ctypes.c_void_p()
        _check(lib.mfa_frame_graph_create(ctx.handle, ctypes.byref(h), ctypes.byref(fd)), "mfa_frame_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib.mfa_frame_graph_launch(self.handle, _stream(stream)), "mfa_frame_graph_launch")

    def close(self):
        if self.handle:
            lib.mfa_frame_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
