"""GB300-native SPIDER: stencils on Sparse Tensor Cores via strided swapping.

The work is done by the CUDA library ``libspider.so`` (C ABI in
``include/spider.h``); this package only marshals arguments to it.  Device
memory and streams come from PyTorch tensors and streams.  There is no
CPU fallback: calls fail when the library or a GPU is missing.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import (SPIDER_BF16X3, SPIDER_BOX, SPIDER_ENGINE_CUDA_CORE, SPIDER_ENGINE_DENSE_TC,
                      SPIDER_ENGINE_SPARSE_TC, SPIDER_ENGINE_SPARSE_TC_COPY, SPIDER_ENGINE_SPARSE_TC_NO_CO, SPIDER_F16X2, SPIDER_STAR, SPIDER_TF32, SpiderError, check)

PRECISIONS = {"tf32": SPIDER_TF32, "f16x2": SPIDER_F16X2, "bf16x3": SPIDER_BF16X3}
ENGINES = {"sparse_tc": SPIDER_ENGINE_SPARSE_TC, "dense_tc": SPIDER_ENGINE_DENSE_TC,
           "cuda_core": SPIDER_ENGINE_CUDA_CORE, "sparse_tc_copy": SPIDER_ENGINE_SPARSE_TC_COPY,
           "sparse_tc_no_co": SPIDER_ENGINE_SPARSE_TC_NO_CO}
SHAPES = {"star": SPIDER_STAR, "box": SPIDER_BOX}


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(int(t.data_ptr()))


class Plan:
    """An owned ``spider_plan`` (see spider_plan_create)."""

    def __init__(self, coeffs, extents, shape: str = "box", precision: str = "tf32", engine: str = "sparse_tc"):
        lib = _native.load()
        w = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float32))
        ext = tuple(int(e) for e in extents)
        r = (w.shape[0] - 1) // 2
        self.extents, self.radius, self.ndim = ext, r, len(ext)
        self.shape_name, self.precision, self.engine = shape, precision, engine
        handle = ctypes.c_void_p()
        check(lib.spider_plan_create(len(ext), (ctypes.c_int64 * len(ext))(*ext), SHAPES[shape], r,
                                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), PRECISIONS[precision],
                                     ctypes.byref(handle)), "spider_plan_create")
        self._h = handle
        if engine != "sparse_tc":
            self.set_engine(engine)

    @property
    def handle(self):
        return self._h

    @property
    def points(self) -> int:
        return int(np.prod(self.extents))

    def set_engine(self, engine: str) -> None:
        check(_native.load().spider_plan_set_engine(self._h, ENGINES[engine]), "spider_plan_set_engine")
        self.engine = engine

    def set_steps_per_pass(self, t: int) -> None:
        check(_native.load().spider_plan_set_steps_per_pass(self._h, int(t)), "spider_plan_set_steps_per_pass")

    def set_tile_variant(self, v: int) -> None:
        check(_native.load().spider_plan_set_tile_variant(self._h, int(v)), "spider_plan_set_tile_variant")

    def autotune(self, grid_in, grid_out, steps: int, stream=None):
        """Times the candidate configurations on these grids and keeps the
        fastest; returns (steps_per_pass, tile_variant)."""
        t, v = ctypes.c_int(), ctypes.c_int()
        check(_native.load().spider_plan_autotune(self._h, _ptr(grid_in), _ptr(grid_out), int(steps),
                                                  _stream_handle(stream), ctypes.byref(t), ctypes.byref(v)),
              "spider_plan_autotune")
        return t.value, v.value

    def autotune_arithmetic(self, grid_in, grid_out, steps: int, err_target: float, stream=None):
        """spider_plan_autotune_arithmetic: the fastest arithmetic whose a
        priori error bound for `steps` steps meets err_target, timed on these
        grids; returns (precision, engine, GStencil/s).  The plan is unchanged."""
        pr, en, rate = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(_native.load().spider_plan_autotune_arithmetic(self._h, _ptr(grid_in), _ptr(grid_out), int(steps),
                                                             float(err_target), _stream_handle(stream),
                                                             ctypes.byref(pr), ctypes.byref(en), ctypes.byref(rate)),
              "spider_plan_autotune_arithmetic")
        prec = {v: k for k, v in PRECISIONS.items()}[pr.value]
        engine = {v: k for k, v in ENGINES.items()}[en.value]
        return prec, engine, rate.value

    def operands(self):
        lib = _native.load()
        na, nm = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib.spider_plan_operands(self._h, None, 0, ctypes.byref(na), None, 0, ctypes.byref(nm)),
              "spider_plan_operands")
        a = np.zeros(na.value, dtype=np.uint32)
        m = np.zeros(nm.value, dtype=np.uint32)
        check(lib.spider_plan_operands(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), a.size, None,
                                       m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), m.size, None),
              "spider_plan_operands")
        return a, m

    def run(self, grid_in, grid_out, steps: int, stream=None) -> None:
        """grid_in / grid_out: contiguous float32 CUDA tensors of the plan's extents."""
        for t in (grid_in, grid_out):
            if not t.is_cuda or not t.is_contiguous() or t.numel() != self.points:
                raise ValueError("grids must be contiguous CUDA tensors of the plan's size")
        check(_native.load().spider_run(self._h, _ptr(grid_in), _ptr(grid_out), int(steps), _stream_handle(stream)),
              "spider_run")

    def run_host(self, host_in: np.ndarray, steps: int, host_out: np.ndarray | None = None, stream=None):
        src = np.ascontiguousarray(host_in, dtype=np.float32)
        if src.size != self.points:
            raise ValueError("host grid has the wrong size")
        out = host_out if host_out is not None else np.empty_like(src)
        check(_native.load().spider_run_host(self._h, src.ctypes.data_as(ctypes.c_void_p),
                                             out.ctypes.data_as(ctypes.c_void_p), int(steps),
                                             _stream_handle(stream)), "spider_run_host")
        return out

    def run_host_async(self, host_in: np.ndarray, steps: int, host_out: np.ndarray, stream=None) -> None:
        """spider_run_host_async: enqueues copy in, steps and copy out and
        returns; host_in and host_out (contiguous float32 arrays of the plan's
        size, pinned for overlap) must stay alive and untouched until sync()."""
        for arr in (host_in, host_out):
            if arr.dtype != np.float32 or not arr.flags.c_contiguous or arr.size != self.points:
                raise ValueError("host grids must be contiguous float32 arrays of the plan's size")
        check(_native.load().spider_run_host_async(self._h, host_in.ctypes.data_as(ctypes.c_void_p),
                                                   host_out.ctypes.data_as(ctypes.c_void_p), int(steps),
                                                   _stream_handle(stream)), "spider_run_host_async")

    def sync(self, stream=None) -> None:
        check(_native.load().spider_plan_sync(self._h, _stream_handle(stream)), "spider_plan_sync")

    def error_bound(self, steps: int, precision: str | None = None, engine: str | None = None) -> float:
        """The library's a priori relative L2 error bound for `steps` steps of
        this stencil in an arithmetic (default: the plan's own)."""
        out = ctypes.c_double()
        check(_native.load().spider_plan_error_bound(self._h, PRECISIONS[precision or self.precision],
                                                     ENGINES[engine or self.engine], int(steps), ctypes.byref(out)),
              "spider_plan_error_bound")
        return out.value

    def device_bytes(self) -> int:
        """Bytes of device memory the plan owns right now."""
        out = ctypes.c_size_t()
        check(_native.load().spider_plan_device_bytes(self._h, ctypes.byref(out)), "spider_plan_device_bytes")
        return out.value

    def close(self) -> None:
        if getattr(self, "_h", None):
            _native.load().spider_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def norms_fp64(a, ref=None, stream=None):
    """(sum a^2, sum ref^2, sum (a-ref)^2, max|a-ref|) computed in FP64 on the GPU."""
    out = (ctypes.c_double * 4)()
    check(_native.load().spider_norms_fp64(_ptr(a), _ptr(ref) if ref is not None else None, int(a.numel()), out,
                                           _stream_handle(stream)), "spider_norms_fp64")
    return tuple(out)


def relative_l2_error(a, ref, stream=None) -> float:
    _, srr, sdd, _ = norms_fp64(a, ref, stream)
    return float(np.sqrt(sdd / srr)) if srr > 0 else float(np.sqrt(sdd))


def constant_check_fp64(a, extents, margin: int, value: float, stream=None) -> float:
    out = ctypes.c_double()
    ext = tuple(int(e) for e in extents)
    check(_native.load().spider_constant_check_fp64(_ptr(a), len(ext), (ctypes.c_int64 * len(ext))(*ext),
                                                    int(margin), float(value), ctypes.byref(out),
                                                    _stream_handle(stream)), "spider_constant_check_fp64")
    return out.value


MMA_KINDS = {"sp_tf32": 0, "sp_f16": 1, "sp_bf16": 2, "dense_tf32": 3}


def measure_mma_rate(kind: str = "sp_tf32", stream=None) -> float:
    """Peak MMAs per second of one warp-level MMA shape on the current GPU
    (spider_measure_mma_rate)."""
    out = ctypes.c_double()
    check(_native.load().spider_measure_mma_rate(MMA_KINDS[kind], ctypes.byref(out), _stream_handle(stream)),
          "spider_measure_mma_rate")
    return out.value


def batch_configure(fuse_min_points: int = 0, queue_steps_per_item: int = 0) -> None:
    """Routing of spider.batch (spider_batch_configure); 0 = default."""
    check(_native.load().spider_batch_configure(int(fuse_min_points), int(queue_steps_per_item)),
          "spider_batch_configure")


def batch(plans, ins, outs, steps, stream=None) -> None:
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    I = (ctypes.c_void_p * n)(*[int(t.data_ptr()) for t in ins])
    O = (ctypes.c_void_p * n)(*[int(t.data_ptr()) for t in outs])
    S = (ctypes.c_int64 * n)(*[int(s) for s in steps])
    check(_native.load().spider_batch(n, P, I, O, S, _stream_handle(stream)), "spider_batch")


class Domain:
    """A plan's grid cut into slabs with ghost planes along its slowest axis
    (spider_domain_create / run / sync); results equal Plan.run bit for bit."""

    def __init__(self, plan: Plan, parts: int, steps_per_exchange: int = 0):
        h = ctypes.c_void_p()
        check(_native.load().spider_domain_create(plan.handle, int(parts), int(steps_per_exchange), ctypes.byref(h)),
              "spider_domain_create")
        self._h = h
        self.parts = int(parts)
        self.points = plan.points

    def slab(self, i: int):
        """(first owned plane, owned planes, ghost planes below, ghost planes above)."""
        v = [ctypes.c_int64() for _ in range(4)]
        check(_native.load().spider_domain_slab(self._h, int(i), *[ctypes.byref(x) for x in v]), "spider_domain_slab")
        return tuple(x.value for x in v)

    def run(self, grid_in, grid_out, steps: int, stream=None) -> None:
        for t in (grid_in, grid_out):
            if not t.is_cuda or not t.is_contiguous() or t.numel() != self.points:
                raise ValueError("grids must be contiguous CUDA tensors of the plan's size")
        check(_native.load().spider_domain_run(self._h, _ptr(grid_in), _ptr(grid_out), int(steps),
                                               _stream_handle(stream)), "spider_domain_run")

    def sync(self, stream=None) -> None:
        check(_native.load().spider_domain_sync(self._h, _stream_handle(stream)), "spider_domain_sync")

    def close(self) -> None:
        if getattr(self, "_h", None):
            _native.load().spider_domain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching stencil server (spider_server_create / submit / poll)."""

    def __init__(self, hbm_budget_bytes: int):
        h = ctypes.c_void_p()
        check(_native.load().spider_server_create(int(hbm_budget_bytes), ctypes.byref(h)), "spider_server_create")
        self._h = h

    def submit(self, plan: Plan, host_in: np.ndarray, steps: int, err_target: float = 1e-3) -> int:
        src = np.ascontiguousarray(host_in, dtype=np.float32)
        if src.size != plan.points:
            raise ValueError("host grid has the wrong size")
        t = ctypes.c_uint64()
        check(_native.load().spider_submit(self._h, plan.handle, src.ctypes.data_as(ctypes.c_void_p), int(steps),
                                           float(err_target), ctypes.byref(t)), "spider_submit")
        return t.value

    def poll(self, ticket: int, out: np.ndarray | None = None):
        """(done, latency_s); when done and `out` is given, the result is copied
        into it and the ticket is released."""
        done, lat = ctypes.c_int(), ctypes.c_double()
        ptr = out.ctypes.data_as(ctypes.c_void_p) if out is not None else None
        check(_native.load().spider_poll(self._h, ctypes.c_uint64(ticket), ptr, ctypes.byref(done),
                                         ctypes.byref(lat)), "spider_poll")
        return bool(done.value), lat.value

    def arithmetic(self, ticket: int):
        """(precision, engine, steps_per_pass, a priori error bound) the server
        chose for a job; valid until poll releases the ticket."""
        p, e, t, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(_native.load().spider_server_job_arithmetic(self._h, ctypes.c_uint64(ticket), ctypes.byref(p),
                                                          ctypes.byref(e), ctypes.byref(t), ctypes.byref(b)),
              "spider_server_job_arithmetic")
        prec = {v: k for k, v in PRECISIONS.items()}[p.value]
        eng = {v: k for k, v in ENGINES.items()}[e.value]
        return prec, eng, t.value, b.value

    def wait(self, timeout_s: float = 0.1):
        """The ticket of a job that finished (each once, in completion order),
        or None if none finished within timeout_s."""
        t, got = ctypes.c_uint64(), ctypes.c_int()
        check(_native.load().spider_server_wait(self._h, float(timeout_s), ctypes.byref(t), ctypes.byref(got)),
              "spider_server_wait")
        return t.value if got.value else None

    def close(self) -> None:
        if getattr(self, "_h", None):
            _native.load().spider_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["Plan", "Domain", "Server", "norms_fp64", "relative_l2_error", "constant_check_fp64", "batch", "SpiderError",
           "measure_mma_rate", "batch_configure",
           "PRECISIONS", "ENGINES", "SHAPES"]
