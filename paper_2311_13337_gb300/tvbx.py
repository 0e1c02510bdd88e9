"""Python binding of the tvbx C-ABI (include/tvbx.h).

Argument marshalling only: every step of the sweep runs in the CUDA library
``lib/libtvbx.so``. Host arrays are numpy arrays; device arrays are CUDA
torch tensors (PyTorch supplies device memory and streams). There is no CPU
fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AXES = ("g", "b_e", "tau_w_e", "E_L_e", "E_L_i", "speed", "a_e", "w_noise",
        "cF_ee", "cF_ei", "cF_ie", "cF_ii")
N_AXES = len(AXES)
MEM_HOST, MEM_DEVICE = 0, 1
SET_NONFINITE, SET_CLAMP_HI, SET_CLAMP_LO, SET_ZERO_VAR, SET_DIVERGED = 1, 2, 4, 8, 16
FC_FP32 = 0
FC_BF16 = 1
FC_BF16X3 = 2
FC_TF32 = 3
FC_TF32X3 = 4
FC_NAMES = {FC_FP32: "fp32", FC_BF16: "bf16", FC_BF16X3: "bf16x3", FC_TF32: "tf32", FC_TF32X3: "tf32x3"}
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NUMERIC", -5: "TIMEOUT",
                -6: "BAD_STATE", -7: "UNSUPPORTED"}
STATE_VARS = ("E", "I", "C_ee", "C_ei", "C_ii", "W_e", "W_i", "OU")


class TvbxError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


class Model(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("g_L", "C_m", "E_e", "E_i", "Q_e", "Q_i", "tau_e", "tau_i",
                 "K_e", "K_i", "N_e", "N_i", "T")] + \
               [("P_e", ctypes.c_double * 10), ("P_i", ctypes.c_double * 10)] + \
               [(n, ctypes.c_double) for n in
                ("mu0", "dmu0", "sig0", "dsig0", "tau0", "dtau0", "rate_floor",
                 "tau_OU", "mu_OU", "sigma_OU", "b_i", "a_i", "tau_w_i",
                 "E_min", "E_max", "E0", "I0", "C_div")] + \
               [("defaults", ctypes.c_double * N_AXES)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name in ("P_e", "P_i", "defaults") else float(v)
        return d


class AxisSpec(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int32), ("n", ctypes.c_int32), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("values", ctypes.POINTER(ctypes.c_double))]


class Grid(ctypes.Structure):
    _fields_ = [("n_axes", ctypes.c_int32), ("axes", ctypes.POINTER(AxisSpec))]


class RunCfg(ctypes.Structure):
    _fields_ = [("dt_ms", ctypes.c_double), ("n_steps", ctypes.c_int64), ("tavg_steps", ctypes.c_int32),
                ("noise_per_set", ctypes.c_int32), ("seed", ctypes.c_uint64), ("p_offset", ctypes.c_int64),
                ("transient_samples", ctypes.c_int32), ("chunk_steps", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("withhold_step", ctypes.c_int32), ("series_mode", ctypes.c_int32),
                ("keep_i_series", ctypes.c_int32)]


class FcCfg(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("fcd_window", ctypes.c_int32), ("fcd_step", ctypes.c_int32),
                ("series_layout", ctypes.c_int32)]


class SurrogateCfg(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("n_hidden", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("n_out", ctypes.c_int32), ("n_members", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("in_lo", ctypes.POINTER(ctypes.c_double)), ("in_hi", ctypes.POINTER(ctypes.c_double))]


_lib = None
EXPORTS = ("tvbx_version", "tvbx_last_error", "tvbx_model_defaults", "tvbx_sweep_create",
           "tvbx_sweep_create_points", "tvbx_sweep_info", "tvbx_run", "tvbx_summary", "tvbx_series",
           "tvbx_series_range", "tvbx_series_pop_range", "tvbx_state", "tvbx_fc", "tvbx_transfer_function", "tvbx_last_kernel",
           "tvbx_launch_count",
           "tvbx_transfer_bytes", "tvbx_profile_enable", "tvbx_profile_read", "tvbx_fc_noalloc", "tvbx_fc_series",
           "tvbx_sweep_destroy", "tvbx_surrogate_create", "tvbx_surrogate_info", "tvbx_surrogate_train",
           "tvbx_surrogate_predict", "tvbx_surrogate_propose", "tvbx_surrogate_rank", "tvbx_surrogate_params", "tvbx_surrogate_gradients",
           "tvbx_surrogate_destroy", "tvbx_fc_pca", "tvbx_fc_pca_project", "tvbx_batch_create", "tvbx_batch_tune",
           "tvbx_batch_run", "tvbx_batch_info", "tvbx_batch_destroy", "tvbx_fc_fitness", "tvbx_top_k",
           "tvbx_series_analysis", "tvbx_bold_defaults", "tvbx_bold", "tvbx_phfcd",
           "tvbx_cell_defaults", "tvbx_cell_rates", "tvbx_tf_fit", "tvbx_tf_refit", "tvbx_run_continue", "tvbx_checkpoint_size",
           "tvbx_checkpoint", "tvbx_restore", "tvbx_set_allocator")


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None   # the installed callbacks, kept alive while installed


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load lib/libtvbx.so (optionally building it first). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"tvbx CUDA library not built: {path} (run paper_2311_13337_gb300/build.py)")
    L = ctypes.CDLL(path)
    vp, i32, i64, dp, fp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
    L.tvbx_version.restype = ctypes.c_char_p
    L.tvbx_last_error.restype = ctypes.c_char_p
    L.tvbx_model_defaults.argtypes = [ctypes.POINTER(Model)]
    L.tvbx_sweep_create.argtypes = [dp, dp, i32, ctypes.POINTER(Grid), ctypes.POINTER(Model), ctypes.POINTER(vp)]
    L.tvbx_sweep_create_points.argtypes = [dp, dp, i32, i64, dp, ctypes.POINTER(Model), ctypes.POINTER(vp)]
    L.tvbx_sweep_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.tvbx_run.argtypes = [vp, ctypes.POINTER(RunCfg), vp]
    L.tvbx_run_continue.argtypes = [vp, i64, i32, vp]
    L.tvbx_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    L.tvbx_checkpoint_size.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
    L.tvbx_checkpoint.argtypes = [vp, vp, ctypes.c_uint64]
    L.tvbx_restore.argtypes = [vp, vp, ctypes.c_uint64]
    L.tvbx_summary.argtypes = [vp, i32, fp, fp, fp, fp, fp]
    L.tvbx_series.argtypes = [vp, i32, fp]
    L.tvbx_series_range.argtypes = [vp, i64, i64, i64, i64, i32, fp]
    L.tvbx_series_pop_range.argtypes = [vp, i32, i64, i64, i64, i64, i32, fp]
    L.tvbx_state.argtypes = [vp, i32, fp]
    L.tvbx_fc.argtypes = [vp, ctypes.POINTER(FcCfg), i32, fp, fp, ctypes.POINTER(i32)]
    L.tvbx_transfer_function.argtypes = [ctypes.POINTER(Model), i32, i64, i32, fp, fp, fp, fp, fp, fp]
    L.tvbx_sweep_destroy.argtypes = [vp]
    L.tvbx_launch_count.restype = ctypes.c_uint64
    L.tvbx_last_kernel.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.tvbx_fc_noalloc.argtypes = [fp, i32, i64, i64, fp, fp, fp, vp]
    L.tvbx_fc_series.argtypes = [fp, i32, i64, i64, ctypes.POINTER(FcCfg), fp, fp, ctypes.POINTER(i32), fp, fp, fp,
                                 vp]
    L.tvbx_surrogate_create.argtypes = [ctypes.POINTER(SurrogateCfg), ctypes.POINTER(vp)]
    L.tvbx_surrogate_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
    L.tvbx_surrogate_train.argtypes = [vp, i32, fp, fp, i64, i32, i32, ctypes.c_float, ctypes.c_float, i32, fp]
    L.tvbx_surrogate_predict.argtypes = [vp, i32, fp, i64, fp, fp]
    L.tvbx_surrogate_propose.argtypes = [vp, i64, ctypes.c_uint64, i32, ctypes.c_float, ctypes.c_float, dp, dp, i32,
                                         fp, fp]
    L.tvbx_surrogate_rank.argtypes = [vp, fp, i64, vp, i32, ctypes.c_float, ctypes.c_float, i32, vp, fp]
    L.tvbx_surrogate_params.argtypes = [vp, i32, fp, fp]
    L.tvbx_surrogate_gradients.argtypes = [vp, i32, fp, fp, i64, ctypes.POINTER(ctypes.c_float), fp]
    L.tvbx_surrogate_destroy.argtypes = [vp]
    L.tvbx_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(RunCfg), i32, ctypes.POINTER(vp)]
    L.tvbx_batch_tune.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i32), fp, ctypes.POINTER(i32)]
    L.tvbx_batch_run.argtypes = [vp]
    L.tvbx_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                  ctypes.POINTER(i32), ctypes.POINTER(i64)]
    L.tvbx_batch_destroy.argtypes = [vp]
    L.tvbx_fc_pca.argtypes = [fp, i32, i64, i32, i32, fp, fp, fp, fp, vp]
    L.tvbx_fc_pca_project.argtypes = [fp, i32, i64, i32, fp, fp, fp, vp]
    L.tvbx_fc_fitness.argtypes = [fp, i64, i32, fp, i32, fp, vp]
    L.tvbx_top_k.argtypes = [fp, i64, i32, fp, fp, vp]
    L.tvbx_series_analysis.argtypes = [fp, i32, i64, i64, ctypes.c_double, fp, ctypes.POINTER(i32), vp]
    L.tvbx_bold_defaults.argtypes = [ctypes.POINTER(BoldParams)]
    L.tvbx_cell_defaults.argtypes = [i32, ctypes.POINTER(CellParams)]
    L.tvbx_cell_rates.argtypes = [ctypes.POINTER(CellParams), i64, dp, dp, dp, i32, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_uint64, dp]
    L.tvbx_tf_fit.argtypes = [ctypes.POINTER(Model), i64, dp, dp, dp, dp, dp, dp, ctypes.POINTER(i32)]
    L.tvbx_tf_refit.argtypes = [ctypes.POINTER(Model), i64, dp, dp, dp, dp, dp, dp, i32, dp,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
    L.tvbx_bold.argtypes = [fp, i32, i64, i64, ctypes.c_double, i32, ctypes.POINTER(BoldParams), fp, i32, fp, vp]
    L.tvbx_phfcd.argtypes = [fp, i32, i64, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, fp,
                             ctypes.POINTER(i32), vp]
    L.tvbx_transfer_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    L.tvbx_profile_enable.argtypes = [vp, i32]
    L.tvbx_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                    ctypes.POINTER(ctypes.c_double)]
    for name in EXPORTS:
        if name not in ("tvbx_version", "tvbx_last_error", "tvbx_launch_count"):
            getattr(L, name).restype = ctypes.c_int32
    _lib = L
    return L


def _check(code: int, where: str):
    if code != 0:
        raise TvbxError(code, where, load().tvbx_last_error().decode())


def version() -> str:
    return load().tvbx_version().decode()


def last_error() -> str:
    return load().tvbx_last_error().decode()


def model_defaults() -> Model:
    m = Model()
    _check(load().tvbx_model_defaults(ctypes.byref(m)), "tvbx_model_defaults")
    return m


def make_model(overrides: dict | None = None) -> Model:
    m = model_defaults()
    for k, v in (overrides or {}).items():
        if k in ("P_e", "P_i"):
            arr = getattr(m, k)
            for i in range(10):
                arr[i] = float(v[i])
        elif k in AXES:
            m.defaults[AXES.index(k)] = float(v)
        else:
            setattr(m, k, float(v))
    return m


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _out_ptr(x):
    """(pointer, mem kind) for a numpy array or a CUDA torch tensor."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("output arrays must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data), MEM_HOST
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("output tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), MEM_DEVICE if x.is_cuda else MEM_HOST
    raise TypeError(f"unsupported array type {type(x)}")


def sweep_create(weights, tract_mm, axes: list, model: Model | None = None):
    """Handle for the Cartesian grid of `axes`: list of (axis name, values) or
    (axis name, (lo, hi, n)); last axis fastest."""
    W, L = _f64(weights), _f64(tract_mm)
    n = W.shape[0]
    specs = (AxisSpec * max(len(axes), 1))()
    keep = []
    for i, (name, vals) in enumerate(axes):
        s = specs[i]
        s.axis = AXES.index(name)
        if isinstance(vals, tuple) and len(vals) == 3 and isinstance(vals[2], int):
            s.lo, s.hi, s.n = float(vals[0]), float(vals[1]), int(vals[2])
            s.values = None
        else:
            arr = _f64(vals)
            keep.append(arr)
            s.n = len(arr)
            s.values = _dptr(arr)
    grid = Grid(len(axes), specs)
    h = ctypes.c_void_p()
    _check(load().tvbx_sweep_create(_dptr(W), _dptr(L), n, ctypes.byref(grid),
                                    ctypes.byref(model) if model is not None else None, ctypes.byref(h)),
           "tvbx_sweep_create")
    return h


def sweep_create_points(weights, tract_mm, params, model: Model | None = None):
    """Handle for explicit points params[n_sets][N_AXES] (axis order AXES)."""
    W, L, P = _f64(weights), _f64(tract_mm), _f64(params).reshape(-1, N_AXES)
    h = ctypes.c_void_p()
    _check(load().tvbx_sweep_create_points(_dptr(W), _dptr(L), W.shape[0], P.shape[0], _dptr(P),
                                           ctypes.byref(model) if model is not None else None, ctypes.byref(h)),
           "tvbx_sweep_create_points")
    return h


def sweep_info(h) -> tuple[int, int, int]:
    p, n, t = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(load().tvbx_sweep_info(h, ctypes.byref(p), ctypes.byref(n), ctypes.byref(t)), "tvbx_sweep_info")
    return p.value, n.value, t.value


KERNEL_AUTO, KERNEL_GENERAL, KERNEL_PREFETCH, KERNEL_DIRECT = 0, 1, 2, 100
SERIES_KEEP, SERIES_STREAM = 0, 1   # tvbx_run_cfg.series_mode
LAYOUT_TNP, LAYOUT_SET4 = 0, 1      # tvbx_fc_cfg.series_layout (tvbx_fc_series)
N_PREFETCH_VARIANTS = 17
PACKED_VARIANTS = (8, 9, 10, 11)   # FP32x2 kernels: need tau_e == tau_i


def _run_cfg(dt_ms=0.1, n_steps=10_000, tavg_steps=10, seed=1, noise_per_set=False, p_offset=0,
             transient_samples=0, chunk_steps=0, kernel=KERNEL_AUTO, withhold_step=0,
             series_mode=SERIES_KEEP, keep_i_series=False) -> RunCfg:
    return RunCfg(float(dt_ms), int(n_steps), int(tavg_steps), int(bool(noise_per_set)), int(seed),
                  int(p_offset), int(transient_samples), int(chunk_steps), int(kernel), int(withhold_step),
                  int(series_mode), int(bool(keep_i_series)))


def run(h, dt_ms=0.1, n_steps=10_000, tavg_steps=10, seed=1, noise_per_set=False, p_offset=0,
        transient_samples=0, chunk_steps=0, stream=None, kernel=KERNEL_AUTO, withhold_step=0,
        series_mode=SERIES_KEEP, keep_i_series=False):
    """Enqueue the integration on `stream` (a torch.cuda.Stream, a raw handle
    or None for the default stream). series_mode SERIES_STREAM keeps one
    chunk of samples and folds it into the FC moments (no series export)."""
    cfg = _run_cfg(dt_ms, n_steps, tavg_steps, seed, noise_per_set, p_offset, transient_samples, chunk_steps,
                   kernel, withhold_step, series_mode, keep_i_series)
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load().tvbx_run(h, ctypes.byref(cfg), sp), "tvbx_run")


def set_allocator(alloc=None, free=None):
    """Install alloc(bytes) -> device pointer (int, 0 on failure) and
    free(pointer) for the handles' device memory (tvbx_set_allocator); no
    arguments restore cudaMalloc / cudaFree."""
    global _allocator_refs
    if alloc is None and free is None:
        _check(load().tvbx_set_allocator(ALLOC_FN(), FREE_FN(), None), "tvbx_set_allocator")
        _allocator_refs = None
        return

    def _a(n, ctx):
        try:
            return int(alloc(int(n))) or None
        except Exception:
            return None

    def _f(p, ctx):
        free(int(p))

    refs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(load().tvbx_set_allocator(refs[0], refs[1], None), "tvbx_set_allocator")
    _allocator_refs = refs


def use_torch_allocator(enable=True):
    """Take the handles' device memory from PyTorch's caching allocator (on
    the current device), so the engine and PyTorch share one pool."""
    if not enable:
        set_allocator()
        return
    import torch
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n), torch.cuda.caching_allocator_delete)


def run_continue(h, n_steps, transient_samples=0, stream=None):
    """Continue the last run for n_steps more steps (tvbx_run_continue)."""
    _check(load().tvbx_run_continue(h, int(n_steps), int(transient_samples), _stream_ptr(stream)),
           "tvbx_run_continue")


def checkpoint(h) -> np.ndarray:
    """The trajectory's checkpoint as a host uint8 array (tvbx_checkpoint)."""
    n = ctypes.c_uint64()
    _check(load().tvbx_checkpoint_size(h, ctypes.byref(n)), "tvbx_checkpoint_size")
    buf = np.zeros(n.value, dtype=np.uint8)
    _check(load().tvbx_checkpoint(h, ctypes.c_void_p(buf.ctypes.data), n.value), "tvbx_checkpoint")
    return buf


def restore(h, buf):
    """Load a checkpoint made by checkpoint() (tvbx_restore)."""
    b = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf,
                             dtype=np.uint8)
    _check(load().tvbx_restore(h, ctypes.c_void_p(b.ctypes.data), b.size), "tvbx_restore")


def summary(h, mean_e_hz=None, mean_i_hz=None, chi=None, mean_fc=None, status=None):
    outs = [mean_e_hz, mean_i_hz, chi, mean_fc, status]
    kinds = {k for _, k in (_out_ptr(o) for o in outs) if k is not None}
    if len(kinds) > 1:
        raise ValueError("summary outputs must all be host or all be device")
    mem = kinds.pop() if kinds else MEM_HOST
    ptrs = [_out_ptr(o)[0] for o in outs]
    _check(load().tvbx_summary(h, mem, *ptrs), "tvbx_summary")


def series(h, out):
    ptr, mem = _out_ptr(out)
    _check(load().tvbx_series(h, mem, ptr), "tvbx_series")


def series_range(h, set_begin, set_count, t_begin, t_count, out, pop=0):
    """Window of the E (pop 0) or I (pop 1, runs with keep_i_series) series."""
    ptr, mem = _out_ptr(out)
    _check(load().tvbx_series_pop_range(h, int(pop), int(set_begin), int(set_count), int(t_begin), int(t_count),
                                        mem, ptr), "tvbx_series_pop_range")


def state(h, out):
    ptr, mem = _out_ptr(out)
    _check(load().tvbx_state(h, mem, ptr), "tvbx_state")


def fc(h, fc_out=None, fcd_out=None, fcd_window=0, fcd_step=0, precision=FC_FP32) -> int:
    kinds = {k for _, k in (_out_ptr(o) for o in (fc_out, fcd_out)) if k is not None}
    if len(kinds) > 1:
        raise ValueError("fc outputs must both be host or both be device")
    mem = kinds.pop() if kinds else MEM_HOST
    cfg = FcCfg(int(precision), int(fcd_window), int(fcd_step))
    nw = ctypes.c_int32()
    _check(load().tvbx_fc(h, ctypes.byref(cfg), mem, _out_ptr(fc_out)[0], _out_ptr(fcd_out)[0],
                          ctypes.byref(nw)), "tvbx_fc")
    return nw.value


def fc_noalloc(series, n_regions: int, n_sets: int, n_samples: int, fc_out, chi=None, mean_fc=None, stream=None):
    """FC with no device allocation (scratch in a fixed array reserved by the
    library). series: CUDA tensor [n_samples][n_regions][n_sets]; outputs are
    CUDA tensors. Calls that overlap on the GPU race; see tvbx.h.

    Every buffer must be a contiguous float32 tensor on the current CUDA
    device holding at least the elements the sizes imply (series
    n_samples * n_regions * n_sets, fc_out n_sets * n_regions^2, chi and
    mean_fc n_sets); anything else raises ValueError before the library is
    called, so a wrong buffer never reaches a kernel."""
    import torch
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    n_regions, n_sets, n_samples = int(n_regions), int(n_sets), int(n_samples)
    need = {"series": n_samples * n_regions * n_sets, "fc_out": n_sets * n_regions * n_regions,
            "chi": n_sets, "mean_fc": n_sets}
    args = []
    for name, x in (("series", series), ("fc_out", fc_out), ("chi", chi), ("mean_fc", mean_fc)):
        if x is None:
            if name in ("series", "fc_out"):
                raise ValueError(f"tvbx_fc_noalloc: {name} is required")
            args.append(None)
            continue
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise ValueError("tvbx_fc_noalloc takes device buffers only (CUDA tensors)")
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError(f"tvbx_fc_noalloc: {name} must be a contiguous float32 tensor")
        if x.device.index != torch.cuda.current_device():
            raise ValueError(f"tvbx_fc_noalloc: {name} is on cuda:{x.device.index}, "
                             f"the current device is cuda:{torch.cuda.current_device()}")
        if x.numel() < need[name]:
            raise ValueError(f"tvbx_fc_noalloc: {name} holds {x.numel()} elements, the sizes need {need[name]}")
        args.append(ctypes.c_void_p(x.data_ptr()))
    _check(load().tvbx_fc_noalloc(args[0], int(n_regions), int(n_sets), int(n_samples), args[1], args[2], args[3],
                                  sp), "tvbx_fc_noalloc")


def fc_series(series, n_regions: int, n_sets: int, n_samples: int, precision=FC_FP32, fc_out=None, fcd_out=None,
              fcd_window=0, fcd_step=0, chi=None, mean_fc=None, set_status=None, stream=None, layout=LAYOUT_TNP) -> int:
    """FC / FCD / chi / mean FC of device series (tvbx_fc_series):
    [n_samples][n_regions][n_sets] (layout LAYOUT_TNP) or set-blocked
    [ceil(n_sets / 4)][n_samples][n_regions][4] (LAYOUT_SET4). Every buffer is a
    CUDA tensor; returns the number of FCD windows. Synchronises the stream."""
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    args = []
    for x in (series, fc_out, fcd_out, chi, mean_fc, set_status):
        if x is None:
            args.append(None)
        else:
            ptr, mem = _out_ptr(x)
            if mem != MEM_DEVICE:
                raise ValueError("tvbx_fc_series takes device buffers only")
            args.append(ptr)
    cfg = FcCfg(int(precision), int(fcd_window), int(fcd_step), int(layout))
    nw = ctypes.c_int32(0)
    _check(load().tvbx_fc_series(args[0], int(n_regions), int(n_sets), int(n_samples), ctypes.byref(cfg), args[1],
                                 args[2], ctypes.byref(nw), args[3], args[4], args[5], sp), "tvbx_fc_series")
    return nw.value


def transfer_function(pop: int, x_e, x_i, W, E_L, C=None, model: Model | None = None) -> np.ndarray:
    """[n][8] = F, F_e, F_i, F_ee, F_ei, F_ii, mu_V, sum_ij C_ij F_ij (the
    integrator's contracted term, 0 without C) from the device code."""
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (x_e, x_i, W, E_L)]
    n = arrs[0].shape[0]
    c = None if C is None else np.ascontiguousarray(C, dtype=np.float32).reshape(n, 3)
    out = np.zeros((n, 8), dtype=np.float32)
    fptr = [ctypes.c_void_p(a.ctypes.data) for a in arrs]
    _check(load().tvbx_transfer_function(ctypes.byref(model) if model is not None else None, int(pop), n,
                                         MEM_HOST, *fptr, ctypes.c_void_p(c.ctypes.data) if c is not None else None,
                                         ctypes.c_void_p(out.ctypes.data)),
           "tvbx_transfer_function")
    return out


KERNEL_NAMES = {KERNEL_GENERAL: "sim_chunk_kernel", KERNEL_DIRECT: "sim_direct_kernel"}
KERNEL_NAMES.update({KERNEL_PREFETCH + v: ("sim_pack_kernel" if v in PACKED_VARIANTS else "sim_tma_kernel" if 12 <= v <= 14 else
                                          "sim_bulk_kernel" if v in (4, 5) else "sim_fast_kernel") + f" (variant {v})"
                     for v in range(N_PREFETCH_VARIANTS)})


def last_kernel(h) -> tuple[int, int]:
    k, pb = ctypes.c_int32(), ctypes.c_int32()
    _check(load().tvbx_last_kernel(h, ctypes.byref(k), ctypes.byref(pb)), "tvbx_last_kernel")
    return k.value, pb.value


def launch_count() -> int:
    return int(load().tvbx_launch_count())


def transfer_bytes(h) -> tuple[int, int]:
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().tvbx_transfer_bytes(h, ctypes.byref(a), ctypes.byref(b)), "tvbx_transfer_bytes")
    return a.value, b.value


def profile_enable(h, enable: bool = True):
    _check(load().tvbx_profile_enable(h, int(bool(enable))), "tvbx_profile_enable")


def profile_read(h) -> tuple[float, int, float]:
    ms, n, rs = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(load().tvbx_profile_read(h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(rs)), "tvbx_profile_read")
    return ms.value, n.value, rs.value


def sweep_destroy(h):
    if h is not None and h.value:
        _check(load().tvbx_sweep_destroy(h), "tvbx_sweep_destroy")


class Sweep:
    """Owning wrapper: one handle, host-side convenience readers."""

    def __init__(self, weights, tract_mm, axes=None, points=None, model: Model | None = None):
        if points is not None:
            self.h = sweep_create_points(weights, tract_mm, points, model)
        else:
            self.h = sweep_create(weights, tract_mm, axes or [], model)
        self.n_sets, self.n_regions, _ = sweep_info(self.h)

    def run(self, **kw):
        run(self.h, **kw)
        self._transient = int(kw.get("transient_samples", 0))
        return self

    def run_continue(self, n_steps, transient_samples=0, stream=None):
        run_continue(self.h, n_steps, transient_samples, stream)
        self._transient = int(transient_samples)
        return self

    def checkpoint(self) -> np.ndarray:
        return checkpoint(self.h)

    def restore(self, buf):
        restore(self.h, buf)
        return self

    @property
    def n_samples(self) -> int:
        return sweep_info(self.h)[2]

    def summary(self) -> dict:
        P = self.n_sets
        out = {k: np.zeros(P, dtype=np.float32) for k in ("mean_e_hz", "mean_i_hz", "chi", "mean_fc")}
        st = np.zeros(P, dtype=np.uint32)
        summary(self.h, out["mean_e_hz"], out["mean_i_hz"], out["chi"], out["mean_fc"], st)
        out["status"] = st
        return out

    def series(self, pop=0) -> np.ndarray:
        """E (pop 0) or I (pop 1, runs with keep_i_series) series [P][N][T]."""
        x = np.zeros((self.n_sets, self.n_regions, self.n_samples), dtype=np.float32)
        if pop == 0:
            series(self.h, x)
        else:
            series_range(self.h, 0, self.n_sets, 0, self.n_samples, x, pop=pop)
        return x

    def series_window(self, set_begin, set_count, t_begin=0, t_count=None) -> np.ndarray:
        if t_count is None:
            t_count = self.n_samples - t_begin
        x = np.zeros((set_count, self.n_regions, t_count), dtype=np.float32)
        series_range(self.h, set_begin, set_count, t_begin, t_count, x)
        return x

    def state(self) -> np.ndarray:
        x = np.zeros((self.n_sets, 8, self.n_regions), dtype=np.float32)
        state(self.h, x)
        return x

    def fc(self, fcd_window=0, fcd_step=0, precision=FC_FP32):
        P, N = self.n_sets, self.n_regions
        out = np.zeros((P, N, N), dtype=np.float32)
        if fcd_window > 0:
            T = self.n_samples - getattr(self, "_transient", 0)
            nw = (T - fcd_window) // fcd_step + 1 if fcd_step > 0 and T >= fcd_window else 1
            fcd_out = np.zeros((P, nw, nw), dtype=np.float32)
            got = fc(self.h, out, fcd_out, fcd_window, fcd_step, precision=precision)
            assert got == nw
            return out, fcd_out
        fc(self.h, out, precision=precision)
        return out

    def close(self):
        sweep_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            if getattr(self, "h", None) is not None:
                self.close()
        except Exception:
            pass


def fc_pca(fc, n_comp=20, n_iter=40, stream=None):
    """Principal components of device FC matrices [P][N][N] (tvbx_fc_pca):
    returns (mean [M], comps [n_comp][M], coef [P][n_comp]) as CUDA tensors and
    the eigenvalues (numpy)."""
    import torch
    P, N = fc.shape[0], fc.shape[1]
    M = N * (N - 1) // 2
    mean = torch.empty(M, dtype=torch.float32, device=fc.device)
    comps = torch.empty((n_comp, M), dtype=torch.float32, device=fc.device)
    coef = torch.empty((P, n_comp), dtype=torch.float32, device=fc.device)
    ev = np.zeros(n_comp, dtype=np.float32)
    sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(load().tvbx_fc_pca(ctypes.c_void_p(fc.data_ptr()), N, P, int(n_comp), int(n_iter),
                              ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(comps.data_ptr()),
                              ctypes.c_void_p(coef.data_ptr()), ctypes.c_void_p(ev.ctypes.data), sp), "tvbx_fc_pca")
    return mean, comps, coef, ev


def fc_pca_project(fc, mean, comps, stream=None):
    import torch
    P, N = fc.shape[0], fc.shape[1]
    coef = torch.empty((P, comps.shape[0]), dtype=torch.float32, device=fc.device)
    sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(load().tvbx_fc_pca_project(ctypes.c_void_p(fc.data_ptr()), N, P, comps.shape[0],
                                      ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(comps.data_ptr()),
                                      ctypes.c_void_p(coef.data_ptr()), sp), "tvbx_fc_pca_project")
    return coef


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def fc_fitness(fc, targets, stream=None):
    """Pearson coefficient of the upper triangles of every FC matrix of
    fc (CUDA [P][N][N]) with every target (CUDA [n_t][N][N] or [N][N])
    (tvbx_fc_fitness): a CUDA tensor [P][n_t] (or [P] for one 2-D target)."""
    import torch
    one = targets.dim() == 2
    tg = targets.reshape(-1, targets.shape[-2], targets.shape[-1]).contiguous()
    fc = fc.contiguous()
    P, N = fc.shape[0], fc.shape[-1]
    out = torch.empty((P, tg.shape[0]), dtype=torch.float32, device=fc.device)
    _check(load().tvbx_fc_fitness(ctypes.c_void_p(fc.data_ptr()), P, N, ctypes.c_void_p(tg.data_ptr()),
                                  tg.shape[0], ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "tvbx_fc_fitness")
    return out[:, 0] if one else out


def top_k(values, k=10, stream=None):
    """The k largest finite entries of a CUDA vector, largest first, ties to
    the lower index (tvbx_top_k): (indices int64, values) CUDA tensors, -1 and
    NaN past the number of finite entries."""
    import torch
    v = values.contiguous().reshape(-1)
    idx = torch.empty(int(k), dtype=torch.int64, device=v.device)
    val = torch.empty(int(k), dtype=torch.float32, device=v.device)
    _check(load().tvbx_top_k(ctypes.c_void_p(v.data_ptr()), v.numel(), int(k), ctypes.c_void_p(idx.data_ptr()),
                             ctypes.c_void_p(val.data_ptr()), _stream_ptr(stream)), "tvbx_top_k")
    return idx, val


AN_FIELDS = ("mean_pli", "psd_fmax", "psd_ampmax", "psd_a", "psd_b", "up_ms", "down_ms", "n_up", "up_samples",
             "n_down", "down_samples")


def series_analysis(series, dt_ms, out=None, stream=None):
    """Table 2 metrics (tvbx_series_analysis) of series [P][N][T] (kHz), a
    CUDA tensor or a host tensor (pinned host memory overlaps its upload
    with the analysis): (CUDA tensor [P][len(AN_FIELDS)], samples used)."""
    import torch
    x = series.contiguous()
    P, N, T = x.shape
    if out is None:
        out = torch.empty((P, len(AN_FIELDS)), dtype=torch.float32, device=x.device if x.is_cuda else "cuda")
    used = ctypes.c_int32(0)
    _check(load().tvbx_series_analysis(ctypes.c_void_p(x.data_ptr()), N, P, T, float(dt_ms),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.byref(used), _stream_ptr(stream)),
           "tvbx_series_analysis")
    return out, used.value


def sweep_analysis(sw, dt_ms, transient_samples=0, batch_sets=4096, stream=None):
    """Table 2 metrics of a sweep's series from sample transient_samples on:
    the series of batch_sets sets at a time are exported to the device
    ([P][N][T]) and analysed. Returns a CUDA tensor [P][len(AN_FIELDS)] and
    the samples used."""
    import torch
    nt = sw.n_samples - int(transient_samples)
    out = torch.empty((sw.n_sets, len(AN_FIELDS)), dtype=torch.float32, device="cuda")
    buf = torch.empty((min(batch_sets, sw.n_sets), sw.n_regions, nt), dtype=torch.float32, device="cuda")
    used = 0
    for p0 in range(0, sw.n_sets, batch_sets):
        m = min(batch_sets, sw.n_sets - p0)
        series_range(sw.h, p0, m, int(transient_samples), nt, buf[:m])
        _, used = series_analysis(buf[:m], dt_ms, out=out[p0:p0 + m], stream=stream)
    return out, used


class BoldParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("kappa", "gamma", "tau", "alpha", "E0", "V0", "theta0", "r0", "TE",
                                               "eps")]


def bold_defaults() -> dict:
    p = BoldParams()
    _check(load().tvbx_bold_defaults(ctypes.byref(p)), "tvbx_bold_defaults")
    return {k: getattr(p, k) for k, _ in BoldParams._fields_}


def bold(series, dt_ms, decim, params=None, state=None, reset_state=True, stream=None):
    """Balloon-Windkessel BOLD (tvbx_bold) of CUDA rates [T][N][P] (kHz):
    a CUDA tensor [T // decim][N][P]; `state` (CUDA [4][N][P]) is read unless
    reset_state and written back."""
    import torch
    x = series.contiguous()
    T, N, P = x.shape
    out = torch.empty((T // int(decim), N, P), dtype=torch.float32, device=x.device)
    pp = None
    if params is not None:
        pp = ctypes.byref(BoldParams(**params))
    st = ctypes.c_void_p(state.data_ptr()) if state is not None else None
    _check(load().tvbx_bold(ctypes.c_void_p(x.data_ptr()), N, P, T, float(dt_ms), int(decim), pp, st,
                            1 if reset_state else 0, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "tvbx_bold")
    return out


def phfcd(bold_series, tr_s, f_lo_hz=0.008, f_hi_hz=0.08, discard=0, stream=None):
    """phFCD (tvbx_phfcd) of CUDA BOLD series [T][N][P]: (CUDA tensor
    [P][T'(T'-1)/2], T')."""
    import torch
    x = bold_series.contiguous()
    T, N, P = x.shape
    n = T
    # T'' (largest 2-3-5-smooth length <= min(T, 8192)) decides the output size
    for m in range(min(T, 8192), 0, -1):
        r = m
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            n = m
            break
    Tp = n - 2 * int(discard)
    out = torch.empty((P, max(Tp * (Tp - 1) // 2, 1)), dtype=torch.float32, device=x.device)
    used = ctypes.c_int32(0)
    _check(load().tvbx_phfcd(ctypes.c_void_p(x.data_ptr()), N, P, T, float(tr_s), float(f_lo_hz), float(f_hi_hz),
                             int(discard), ctypes.c_void_p(out.data_ptr()), ctypes.byref(used), _stream_ptr(stream)),
           "tvbx_phfcd")
    return out, used.value


class CellParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("C", "gL", "EL", "VT", "Delta", "Vreset", "t_ref", "Qe", "Qi", "tau_e",
                                               "tau_i", "Ee", "Ei", "Ke", "Ki")]


def cell_defaults(pop: int = 0) -> dict:
    """Regular-spiking (0) or fast-spiking (1) AdEx cell (tvbx_cell_defaults)."""
    p = CellParams()
    _check(load().tvbx_cell_defaults(int(pop), ctypes.byref(p)), "tvbx_cell_defaults")
    return {k: getattr(p, k) for k, _ in CellParams._fields_}


def cell_rates(cell: dict, nu_e_khz, nu_i_khz, W_pA, n_cells=16, T_ms=5000.0, transient_ms=200.0, dt_ms=0.05,
               seed=1) -> np.ndarray:
    """Output rates (kHz) of single AdEx cells with Poisson inputs (tvbx_cell_rates)."""
    arrs = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (nu_e_khz, nu_i_khz, W_pA)]
    out = np.zeros(arrs[0].size)
    _check(load().tvbx_cell_rates(ctypes.byref(CellParams(**cell)), arrs[0].size, _dptr(arrs[0]), _dptr(arrs[1]),
                                  _dptr(arrs[2]), int(n_cells), float(T_ms), float(transient_ms), float(dt_ms),
                                  int(seed), _dptr(out)), "tvbx_cell_rates")
    return out


def tf_refit(nu_e_khz, nu_i_khz, W_pA, E_L, rate_khz, P_init, max_iter=200, model: Model | None = None):
    """Second stage of the Table 1 fit (tvbx_tf_refit): least squares on the
    rates from P_init: (P[10], rms rate error in kHz, points used)."""
    m = model if model is not None else make_model()
    arrs = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (nu_e_khz, nu_i_khz, W_pA, E_L,
                                                                               rate_khz)]
    P0 = np.ascontiguousarray(P_init, dtype=np.float64)
    if P0.shape != (10,):
        raise ValueError("P_init must have 10 coefficients")
    P = np.zeros(10)
    rms = ctypes.c_double(0.0)
    used = ctypes.c_int32(0)
    _check(load().tvbx_tf_refit(ctypes.byref(m), arrs[0].size, *[_dptr(a) for a in arrs], _dptr(P0), int(max_iter),
                                _dptr(P), ctypes.byref(rms), ctypes.byref(used)), "tvbx_tf_refit")
    return P, rms.value, used.value


def tf_fit(nu_e_khz, nu_i_khz, W_pA, E_L, rate_khz, model: Model | None = None):
    """Table 1 coefficients fitted to measured rates (tvbx_tf_fit): (P[10], points used)."""
    m = model if model is not None else make_model()
    arrs = [np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64) for a in (nu_e_khz, nu_i_khz, W_pA, E_L,
                                                                               rate_khz)]
    P = np.zeros(10)
    used = ctypes.c_int32(0)
    _check(load().tvbx_tf_fit(ctypes.byref(m), arrs[0].size, *[_dptr(a) for a in arrs], _dptr(P), ctypes.byref(used)),
           "tvbx_tf_fit")
    return P, used.value


class Surrogate:
    """Ensemble MLP surrogate (tvbx_surrogate_*): parameters -> summary
    statistics, trained and evaluated by the library's CUDA kernels."""

    def __init__(self, lo, hi, n_out, n_hidden=256, n_layers=3, n_members=4, seed=1):
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.n_in, self.n_out = lo.size, int(n_out)
        cfg = SurrogateCfg(self.n_in, int(n_hidden), int(n_layers), self.n_out, int(n_members), int(seed),
                           _dptr(lo), _dptr(hi))
        self.h = ctypes.c_void_p()
        _check(load().tvbx_surrogate_create(ctypes.byref(cfg), ctypes.byref(self.h)), "tvbx_surrogate_create")
        n, e = ctypes.c_int64(), ctypes.c_int32()
        _check(load().tvbx_surrogate_info(self.h, ctypes.byref(n), ctypes.byref(e)), "tvbx_surrogate_info")
        self.n_params, self.n_members = n.value, e.value
        self.dims = [self.n_in] + [int(n_hidden)] * int(n_layers) + [self.n_out]

    def _ptr(self, a, cols):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr()), (MEM_DEVICE if a.is_cuda else MEM_HOST), a.shape[0], a
        a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1, cols)
        return ctypes.c_void_p(a.ctypes.data), MEM_HOST, a.shape[0], a

    def train(self, X, Y, epochs=1, batch=1024, lr=1e-3, weight_decay=1e-4, shuffle=True, keep_scale=False):
        """keep_scale: keep the output standardisation of the earlier
        training call (fine-tuning) instead of recomputing it from Y."""
        px, mx, n, kx = self._ptr(X, self.n_in)
        py, my, _, ky = self._ptr(Y, self.n_out)
        if mx != my:
            raise ValueError("X and Y must both be host or both be device arrays")
        losses = np.zeros(int(epochs), dtype=np.float32)
        _check(load().tvbx_surrogate_train(self.h, mx, px, py, n, int(epochs), int(batch), float(lr),
                                           float(weight_decay), (1 if shuffle else 0) | (2 if keep_scale else 0),
                                           ctypes.c_void_p(losses.ctypes.data)), "tvbx_surrogate_train")
        return losses

    def predict(self, X, want_var=False):
        px, mx, n, kx = self._ptr(X, self.n_in)
        if mx == MEM_DEVICE:
            import torch
            mean = torch.empty((n, self.n_out), dtype=torch.float32, device=X.device)
            var = torch.empty((n, self.n_out), dtype=torch.float32, device=X.device) if want_var else None
            pm, pv = ctypes.c_void_p(mean.data_ptr()), (ctypes.c_void_p(var.data_ptr()) if want_var else None)
        else:
            mean = np.zeros((n, self.n_out), dtype=np.float32)
            var = np.zeros((n, self.n_out), dtype=np.float32) if want_var else None
            pm, pv = ctypes.c_void_p(mean.ctypes.data), (ctypes.c_void_p(var.ctypes.data) if want_var else None)
        _check(load().tvbx_surrogate_predict(self.h, mx, px, n, pm, pv), "tvbx_surrogate_predict")
        return (mean, var) if want_var else mean

    def propose(self, n_candidates, n_propose, output, threshold, var_weight=1.0, round=0, box=None):
        """box: optional (lo, hi) candidate box; lo[i] == hi[i] fixes input i."""
        pts = np.zeros((int(n_propose), self.n_in), dtype=np.float32)
        sc = np.zeros(int(n_propose), dtype=np.float32)
        lo = hi = None
        if box is not None:
            lo, hi = (np.ascontiguousarray(b, dtype=np.float64) for b in box)
        _check(load().tvbx_surrogate_propose(self.h, int(n_candidates), int(round), int(output), float(threshold),
                                             float(var_weight), _dptr(lo) if lo is not None else None,
                                             _dptr(hi) if hi is not None else None, int(n_propose),
                                             ctypes.c_void_p(pts.ctypes.data), ctypes.c_void_p(sc.ctypes.data)),
               "tvbx_surrogate_propose")
        return pts, sc

    def rank(self, X, n_propose, output, threshold, var_weight=1.0, exclude=None):
        """Indices (best first) and scores of the n_propose best rows of the
        host candidates X by the proposal score; rows where exclude (bool
        [n]) is set are never chosen."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != self.n_in:
            raise ValueError(f"X must be [n][{self.n_in}]")
        ex = None
        if exclude is not None:
            ex = np.ascontiguousarray(exclude, dtype=np.uint8)
            if ex.shape != (X.shape[0],):
                raise ValueError("exclude must have one entry per candidate")
        idx = np.zeros(int(n_propose), dtype=np.int64)
        sc = np.zeros(int(n_propose), dtype=np.float32)
        _check(load().tvbx_surrogate_rank(self.h, ctypes.c_void_p(X.ctypes.data), X.shape[0],
                                          ctypes.c_void_p(ex.ctypes.data) if ex is not None else None, int(output),
                                          float(threshold), float(var_weight), int(n_propose),
                                          ctypes.c_void_p(idx.ctypes.data), ctypes.c_void_p(sc.ctypes.data)),
               "tvbx_surrogate_rank")
        return idx, sc

    def params(self, member=0) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().tvbx_surrogate_params(self.h, int(member), ctypes.c_void_p(out.ctypes.data), None),
               "tvbx_surrogate_params")
        return out

    def set_params(self, vec, member=0):
        v = np.ascontiguousarray(vec, dtype=np.float32)
        assert v.size == self.n_params
        _check(load().tvbx_surrogate_params(self.h, int(member), None, ctypes.c_void_p(v.ctypes.data)),
               "tvbx_surrogate_params")

    def gradients(self, X, Y, member=0):
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().tvbx_surrogate_gradients(self.h, int(member), ctypes.c_void_p(X.ctypes.data),
                                               ctypes.c_void_p(Y.ctypes.data), X.shape[0], ctypes.byref(loss),
                                               ctypes.c_void_p(g.ctypes.data)), "tvbx_surrogate_gradients")
        return loss.value, g

    def close(self):
        if self.h is not None and self.h.value:
            _check(load().tvbx_surrogate_destroy(self.h), "tvbx_surrogate_destroy")
            self.h = None


class Batch:
    """Several sweeps run as one persistent launch in a CUDA graph
    (tvbx_batch_*). jobs: list of (Sweep, dict of run settings)."""

    def __init__(self, jobs):
        self.sweeps = [sw for sw, _ in jobs]
        handles = (ctypes.c_void_p * len(jobs))(*[sw.h.value for sw in self.sweeps])
        cfgs = (RunCfg * len(jobs))(*[_run_cfg(**kw) for _, kw in jobs])
        self._keep = (handles, cfgs)
        self.h = ctypes.c_void_p()
        _check(load().tvbx_batch_create(ctypes.cast(handles, ctypes.POINTER(ctypes.c_void_p)), cfgs, len(jobs),
                                        ctypes.byref(self.h)), "tvbx_batch_create")
        for sw, kw in jobs:
            sw._transient = int(kw.get("transient_samples", 0))

    def tune(self, trial_steps=200):
        t, k, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = np.zeros(16, dtype=np.float32)
        _check(load().tvbx_batch_tune(self.h, int(trial_steps), ctypes.byref(t), ctypes.byref(k),
                                      ctypes.c_void_p(ms.ctypes.data), ctypes.byref(n)), "tvbx_batch_tune")
        return t.value, k.value, ms[:n.value]

    def run(self):
        _check(load().tvbx_batch_run(self.h), "tvbx_batch_run")
        return self

    def info(self) -> dict:
        t, k, g = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        n, nodes = ctypes.c_int64(), ctypes.c_int64()
        _check(load().tvbx_batch_info(self.h, ctypes.byref(t), ctypes.byref(k), ctypes.byref(n), ctypes.byref(g),
                                      ctypes.byref(nodes)), "tvbx_batch_info")
        return {"threads": t.value, "smem_kb": k.value, "items": n.value, "grid": g.value, "graph_nodes": nodes.value}

    def close(self):
        if self.h is not None and self.h.value:
            _check(load().tvbx_batch_destroy(self.h), "tvbx_batch_destroy")
            self.h = None
