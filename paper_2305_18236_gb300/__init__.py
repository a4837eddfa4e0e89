"""GEMM for one NVIDIA GB300 (sm_103a): C = alpha * op(A) op(B) + beta * C.

A from-scratch, GPU-native form of the layered GEMM of Kuzma et al.,
"Fast Matrix Multiplication via Compiler-only Layered Data Reorganization
and Intrinsic Lowering" (SPE 2023): blocking and packing become TMA tile
loads into a shared-memory ring and a persistent tile scheduler; the
matrix-engine micro kernel becomes tcgen05 MMAs into tensor memory.  Modes:
FP32 SIMT, plain BF16 tensor cores, and 3xBF16 split precision.

The compute lives in ``_build/libgb300gemm.so`` (C ABI: ``include/gemm.h``),
built by :func:`build.build`; importing this package does not load it.
"""
from . import inputs  # noqa: F401  (seeded synthetic matrices; no CUDA)

__all__ = ["inputs", "build_library", "matmul", "matmul_bf16", "split_bf16", "gemm_from_host",
           "gemm_backward", "gemm_grouped", "GroupedPlan", "GemmFn", "Gemm", "handle", "sync",
           "syr2k"]


def build_library(force=False):
    from .build import build

    return build(force=force)


def __getattr__(name):
    # Torch-facing API is imported lazily so that `inputs` stays usable
    # without torch's CUDA initialisation.
    if name in ("matmul", "matmul_bf16", "split_bf16", "gemm_from_host", "gemm_backward",
                "gemm_grouped", "GroupedPlan", "GemmFn", "Gemm", "handle", "sync", "syr2k"):
        from . import gemm as _g

        return getattr(_g, name)
    raise AttributeError(name)
