"""Torch-facing wrappers over the C ABI (``include/gemm.h``).

Thin marshalling only: tensors are turned into (pointer, ld) pairs and the
current torch stream is passed through; the library's kernels do all the
work.  PyTorch provides device memory (tensors, the workspace) and streams.

    import paper_2305_18236_gb300 as g
    C = g.matmul(A, B, mode="bf16x3")                  # C = A @ B
    g.matmul(A, B, C=C, alpha=1.5, beta=0.5)           # C = 1.5 A B + 0.5 C
    Y = g.GemmFn.apply(X, W, "bf16x3")                 # differentiable X @ W
"""
import ctypes

import torch

from . import _lib
from ._lib import (LAYOUTS, MODES, SPLIT_PLACES, SPLITK_REDUCES, check, gemm_config_t,
                   gemm_problem_t)

__all__ = ["Gemm", "handle", "matmul", "matmul_bf16", "split_bf16", "gemm_from_host",
           "gemm_backward", "gemm_grouped", "GroupedPlan", "GemmFn", "sync"]


def _mode(mode):
    if isinstance(mode, int):
        return mode
    return MODES[mode]


def _ld(t):
    """Row stride of a 2-D row-major tensor (last dim contiguous)."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    if t.numel() == 0:
        return max(1, t.size(1))  # nothing is read or written: any valid stride
    if t.size(1) > 1 and t.stride(1) != 1:
        raise ValueError("the last dimension must be contiguous (row-major storage)")
    return t.stride(0) if t.size(0) > 1 else max(1, t.size(1))


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Gemm:
    """A library handle bound to one CUDA device, plus a torch-allocated
    workspace that grows on demand.  Use one handle per stream."""

    def __init__(self, device=None):
        self.lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.gemm_create(ctypes.byref(h)), "gemm_create")
        self.h = h
        self._ws = None
        self._ws_sizes = {}  # (mode, transA, transB, M, N, K) -> bytes, for this config

    def close(self):
        if self.h:
            self.lib.gemm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration -------------------------------------------------
    def set_config(self, bn=0, bk=0, stages=0, split_k=0, raster_group=0, max_ctas=0,
                   promote_k=0, cta_group=0, wait_poll_limit=0, operand_layout="auto",
                   split_place="auto", splitk_reduce="auto"):
        """operand_layout: "auto" (library choice), "as_stored" (MN-major tiles
        for operands stored K x rows) or "k_major" (every operand made
        K-contiguous first).  split_place (3xBF16): "auto", "prepass" (split
        pass before the kernel), "in_kernel" (the kernel splits FP32 tiles
        in shared memory), "in_kernel_a" / "in_kernel_b" (the kernel splits
        A / B, the pass the other; matmul only).  splitk_reduce: "auto" (split-K
        slices added inside the GEMM kernel where a cluster can hold them) or
        "launch" (a second kernel adds them); the same bits either way."""
        layout = LAYOUTS[operand_layout] if isinstance(operand_layout, str) else operand_layout
        place = SPLIT_PLACES[split_place] if isinstance(split_place, str) else split_place
        red = SPLITK_REDUCES[splitk_reduce] if isinstance(splitk_reduce, str) else splitk_reduce
        cfg = gemm_config_t(bn, bk, stages, split_k, raster_group, max_ctas, promote_k, cta_group,
                            wait_poll_limit, layout, place, red)
        check(self.lib.gemm_set_config(self.h, ctypes.byref(cfg)), "gemm_set_config", self.h)
        self._ws_sizes.clear()

    def reset_config(self):
        check(self.lib.gemm_set_config(self.h, None), "gemm_set_config", self.h)
        self._ws_sizes.clear()

    def ensure_workspace(self, nbytes):
        if nbytes == 0:
            return
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            check(self.lib.gemm_set_workspace(self.h, ctypes.c_void_p(self._ws.data_ptr()),
                                              self._ws.numel()), "gemm_set_workspace", self.h)

    def workspace_size(self, mode, transA, transB, M, N, K):
        key = (_mode(mode), bool(transA), bool(transB), M, N, K)
        n = self._ws_sizes.get(key)
        if n is None:
            n = self.lib.gemm_workspace_size(self.h, key[0], int(transA), int(transB), M, N, K)
            if len(self._ws_sizes) > 4096:
                self._ws_sizes.clear()
            self._ws_sizes[key] = n
        return n

    def last_launch_count(self):
        return self.lib.gemm_last_launch_count(self.h)

    def last_error_arg(self):
        return self.lib.gemm_last_error_arg(self.h)

    # -- raw C-ABI calls (device pointers as ints) ----------------------
    def gemm(self, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, mode,
             stream=None):
        """The C-ABI gemm() with raw device pointers; returns the status."""
        s = _stream(self.device) if stream is None else ctypes.c_void_p(stream)
        return self.lib.gemm(self.h, int(transA), int(transB), M, N, K, alpha,
                             ctypes.c_void_p(A), lda, ctypes.c_void_p(B), ldb, beta,
                             ctypes.c_void_p(C), ldc, _mode(mode), s)

    def sync(self, stream=None):
        s = _stream(self.device) if stream is None else ctypes.c_void_p(stream)
        return self.lib.gemm_sync(self.h, s)


_HANDLES = {}


def handle(device=None):
    """The shared handle of a device (created on first use)."""
    idx = torch.cuda.current_device() if device is None else (torch.device(device).index or 0)
    if idx not in _HANDLES:
        _HANDLES[idx] = Gemm(idx)
    return _HANDLES[idx]


def _dims(A, B, transA, transB):
    M, K = (A.size(1), A.size(0)) if transA else (A.size(0), A.size(1))
    Kb, N = (B.size(1), B.size(0)) if transB else (B.size(0), B.size(1))
    if K != Kb:
        raise ValueError("inner dimensions differ: %d vs %d" % (K, Kb))
    return M, N, K


def _out(C, M, N, beta, device):
    if C is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
        C = torch.empty((M, N), dtype=torch.float32, device=device)
    if C.dtype != torch.float32 or tuple(C.shape) != (M, N):
        raise ValueError("C must be float32 of shape (%d, %d)" % (M, N))
    return C


def matmul(A, B, C=None, alpha=1.0, beta=0.0, transA=False, transB=False, mode="bf16x3",
           h=None):
    """C = alpha * op(A) @ op(B) + beta * C for float32 CUDA tensors (in place
    into C when given).  mode: 'f32_simt', 'bf16' or 'bf16x3'."""
    if A.dtype == torch.bfloat16 or B.dtype == torch.bfloat16:
        return matmul_bf16(A, B, C, alpha, beta, transA, transB, h)
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError("float32 (or bfloat16) inputs expected")
    h = h or handle(A.device)
    M, N, K = _dims(A, B, transA, transB)
    C = _out(C, M, N, beta, A.device)
    m = _mode(mode)
    h.ensure_workspace(h.workspace_size(m, transA, transB, M, N, K))
    st = h.gemm(int(transA), int(transB), M, N, K, float(alpha), A.data_ptr(), _ld(A),
                B.data_ptr(), _ld(B), float(beta), C.data_ptr(), _ld(C), m)
    check(st, "gemm", h.h)
    return C


def syr2k(A, B, C=None, alpha=1.0, beta=0.0, uplo="lower", trans=False, mode="bf16x3", h=None):
    """SYR2K (Section 5.1): the ``uplo`` triangle of C <- alpha (A B^T + B A^T)
    + beta C for float32 CUDA tensors A, B of shape (N, K), or alpha (A^T B +
    B^T A) + beta C for shape (K, N) with ``trans``.  The other triangle of C
    is left as it is (uninitialised when C is None)."""
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise TypeError("float32 inputs expected")
    if tuple(A.shape) != tuple(B.shape):
        raise ValueError("A and B must have the same shape")
    h = h or handle(A.device)
    N, K = (A.size(1), A.size(0)) if trans else (A.size(0), A.size(1))
    C = _out(C, N, N, beta, A.device)
    m = _mode(mode)
    h.ensure_workspace(h.lib.gemm_syr2k_workspace_size(h.h, m, int(trans), N, K))
    st = h.lib.gemm_syr2k(h.h, _lib.UPLOS[uplo], int(trans), N, K, float(alpha),
                          ctypes.c_void_p(A.data_ptr()), _ld(A), ctypes.c_void_p(B.data_ptr()),
                          _ld(B), float(beta), ctypes.c_void_p(C.data_ptr()), _ld(C), m,
                          _stream(A.device))
    check(st, "gemm_syr2k", h.h)
    return C


def matmul_bf16(A, B, C=None, alpha=1.0, beta=0.0, transA=False, transB=False, h=None):
    """C = alpha * op(A) @ op(B) + beta * C for bfloat16 A, B and float32 C."""
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16:
        raise TypeError("bfloat16 inputs expected")
    h = h or handle(A.device)
    M, N, K = _dims(A, B, transA, transB)
    C = _out(C, M, N, beta, A.device)
    h.ensure_workspace(h.workspace_size(MODES["bf16"], transA, transB, M, N, K))
    st = h.lib.gemm_bf16(h.h, int(transA), int(transB), M, N, K, float(alpha),
                         ctypes.c_void_p(A.data_ptr()), _ld(A), ctypes.c_void_p(B.data_ptr()),
                         _ld(B), float(beta), ctypes.c_void_p(C.data_ptr()), _ld(C),
                         _stream(A.device))
    check(st, "gemm_bf16", h.h)
    return C


def split_bf16(X, trans=False, with_lo=True, h=None):
    """(hi, lo) bfloat16 tensors of op(X) (lo None when with_lo is False)."""
    h = h or handle(X.device)
    rows, cols = (X.size(1), X.size(0)) if trans else (X.size(0), X.size(1))
    ldo = (cols + 7) // 8 * 8
    hi = torch.empty((rows, ldo), dtype=torch.bfloat16, device=X.device)
    lo = torch.empty((rows, ldo), dtype=torch.bfloat16, device=X.device) if with_lo else None
    st = h.lib.gemm_split_bf16(h.h, int(trans), rows, cols, ctypes.c_void_p(X.data_ptr()), _ld(X),
                               ctypes.c_void_p(hi.data_ptr()),
                               ctypes.c_void_p(lo.data_ptr() if lo is not None else 0), ldo,
                               _stream(X.device))
    check(st, "gemm_split_bf16", h.h)
    return hi[:, :cols], (lo[:, :cols] if lo is not None else None)


def gemm_from_host(A, B, C=None, alpha=1.0, beta=0.0, transA=False, transB=False,
                   mode="bf16x3", h=None, stream=None):
    """gemm_from_host on CPU float32 tensors (pinned for asynchronous copies);
    C (CPU) is updated in place and returned."""
    h = h or handle()
    M, N, K = _dims(A, B, transA, transB)
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, pin_memory=A.is_pinned())
    h.ensure_workspace(h.workspace_size(_mode(mode), transA, transB, M, N, K))
    s = _stream(h.device) if stream is None else ctypes.c_void_p(stream)
    st = h.lib.gemm_from_host(h.h, int(transA), int(transB), M, N, K, float(alpha),
                              ctypes.c_void_p(A.data_ptr()), _ld(A),
                              ctypes.c_void_p(B.data_ptr()), _ld(B), float(beta),
                              ctypes.c_void_p(C.data_ptr()), _ld(C), _mode(mode), s)
    check(st, "gemm_from_host", h.h)
    return C


def gemm_backward(dC, A, B, transA=False, transB=False, need_dA=True, need_dB=True,
                  mode="bf16x3", h=None):
    """(dA, dB) of C = op(A) op(B) for the given dC (stored like A and B)."""
    h = h or handle(dC.device)
    M, N, K = _dims(A, B, transA, transB)
    dA = torch.empty_like(A) if need_dA else None
    dB = torch.empty_like(B) if need_dB else None
    m = _mode(mode)
    h.ensure_workspace(max(h.workspace_size(m, 0, 0, M, K, N), h.workspace_size(m, 0, 0, K, N, M)))
    st = h.lib.gemm_backward(h.h, int(transA), int(transB), M, N, K,
                             ctypes.c_void_p(dC.data_ptr()), _ld(dC),
                             ctypes.c_void_p(A.data_ptr()), _ld(A),
                             ctypes.c_void_p(B.data_ptr()), _ld(B),
                             ctypes.c_void_p(dA.data_ptr() if dA is not None else 0),
                             _ld(dA) if dA is not None else 1,
                             ctypes.c_void_p(dB.data_ptr() if dB is not None else 0),
                             _ld(dB) if dB is not None else 1, m, _stream(dC.device))
    check(st, "gemm_backward", h.h)
    return dA, dB


def _problem_array(problems):
    arr = (gemm_problem_t * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        A, B, C = p["A"], p["B"], p["C"]
        tA, tB = int(p.get("transA", False)), int(p.get("transB", False))
        M, N, K = _dims(A, B, tA, tB)
        arr[i] = gemm_problem_t(M, N, K, _ld(A), _ld(B), _ld(C), A.data_ptr(), B.data_ptr(),
                                C.data_ptr(), float(p.get("alpha", 1.0)),
                                float(p.get("beta", 0.0)), tA, tB)
        keep.append((A, B, C))
    return arr, keep


class GroupedPlan:
    """gemm_grouped_plan_*: many independent GEMMs (dicts with A, B, C CUDA
    tensors and optional alpha, beta, transA, transB) run as one split launch
    plus one persistent tensor-core launch.  autotune: time the candidate
    configurations at creation; graph: capture the launches in a CUDA graph
    on the first run and replay it."""

    def __init__(self, problems, mode="bf16x3", autotune=False, graph=False, h=None,
                 stream=None):
        self.h = h or handle(problems[0]["A"].device if problems else None)
        self.lib = self.h.lib
        self._arr, self._keep = _problem_array(problems)
        flags = (_lib.GROUPED_AUTOTUNE if autotune else 0) | (_lib.GROUPED_GRAPH if graph else 0)
        s = _stream(self.h.device) if stream is None else ctypes.c_void_p(stream)
        plan = ctypes.c_void_p()
        st = self.lib.gemm_grouped_plan_create(self.h.h, _mode(mode), self._arr, len(problems),
                                               flags, s, ctypes.byref(plan))
        check(st, "gemm_grouped_plan_create", self.h.h)
        self.plan = plan

    def run(self, stream=None):
        s = _stream(self.h.device) if stream is None else ctypes.c_void_p(stream)
        check(self.lib.gemm_grouped_plan_run(self.plan, s), "gemm_grouped_plan_run", self.h.h)

    def config(self):
        cfg = gemm_config_t()
        ms = ctypes.c_double()
        check(self.lib.gemm_grouped_plan_config(self.plan, ctypes.byref(cfg), ctypes.byref(ms)),
              "gemm_grouped_plan_config")
        names = {v: k for k, v in LAYOUTS.items()}
        places = {v: k for k, v in SPLIT_PLACES.items()}
        return {"bn": cfg.bn, "bk": cfg.bk, "stages": cfg.stages, "split_k": cfg.split_k,
                "raster_group": cfg.raster_group, "cta_group": cfg.cta_group,
                "operand_layout": names.get(cfg.operand_layout, cfg.operand_layout),
                "split_place": places.get(cfg.split_place, cfg.split_place),
                "tuned_ms": ms.value}

    def close(self):
        if self.plan:
            self.lib.gemm_grouped_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm_grouped(problems, mode="bf16x3", h=None):
    """One-shot grouped GEMM (builds, runs and frees a plan; synchronises)."""
    h = h or handle()
    arr, keep = _problem_array(problems)
    st = h.lib.gemm_grouped(h.h, _mode(mode), arr, len(problems), _stream(h.device))
    check(st, "gemm_grouped", h.h)


def sync(h=None):
    """gemm_sync on the current stream: raises GemmError on a kernel timeout."""
    h = h or handle()
    check(h.sync(), "gemm_sync", h.h)


class GemmFn(torch.autograd.Function):
    """Y = X @ W with the library's forward and hand-written backward
    (dX = dY W^T, dW = X^T dY, both through gemm_backward)."""

    @staticmethod
    def forward(ctx, X, W, mode="bf16x3"):
        ctx.save_for_backward(X, W)
        ctx.mode = mode
        return matmul(X.contiguous(), W.contiguous(), mode=mode)

    @staticmethod
    def backward(ctx, dY):
        X, W = ctx.saved_tensors
        dX, dW = gemm_backward(dY.contiguous().float(), X.contiguous(), W.contiguous(),
                               need_dA=ctx.needs_input_grad[0], need_dB=ctx.needs_input_grad[1],
                               mode=ctx.mode)
        return dX, dW, None
