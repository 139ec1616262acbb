"""Device-side twin of ``datagen``: the same recipes, generated by the CUDA
generator in ``libtqpgen.so`` straight into device memory (bit-identical to
the host generator).  Holds no query-operator arithmetic."""
from __future__ import annotations

import ctypes
import os

import torch

from . import datagen as dg

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtqpgen.so")
if not os.path.exists(_PATH):
    raise ImportError(f"libtqpgen.so not built ({_PATH}); run python -m paper_2209_04579_b300.build")
_lib = ctypes.CDLL(_PATH)


class _Recipe(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dtype", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("key_seed", ctypes.c_uint64), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64),
                ("mul", ctypes.c_int64), ("m", ctypes.c_int64), ("noise_p32", ctypes.c_uint64),
                ("seed2", ctypes.c_uint64)]


_lib.tqpgen_column.argtypes = [ctypes.POINTER(_Recipe), ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
_lib.tqpgen_column.restype = ctypes.c_int

_TORCH = {1: torch.int8, 2: torch.int16, 3: torch.int32, 4: torch.int64}
_M64 = (1 << 64) - 1


def generate(rec: dg.Recipe, n: int, start: int = 0, zipf: torch.Tensor | None = None,
             out: torch.Tensor | None = None, device="cuda") -> torch.Tensor:
    out = torch.empty(n, dtype=_TORCH[rec.dtype], device=device) if out is None else out
    r = _Recipe(rec.kind, rec.dtype, rec.seed & _M64, rec.key_seed & _M64, rec.lo, rec.hi, rec.mul, rec.m,
                rec.noise_p32, rec.seed2 & _M64)
    zp = zipf.data_ptr() if zipf is not None else 0
    zn = zipf.numel() if zipf is not None else 0
    st = _lib.tqpgen_column(ctypes.byref(r), start, n, ctypes.c_void_p(out.data_ptr() if n else 0),
                            ctypes.c_void_p(zp), zn, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError(f"tqpgen_column failed with status {st}")
    return out


def make_table(recipes: dict, n: int, start: int = 0, zipf: torch.Tensor | None = None, device="cuda") -> dict:
    return {name: generate(r, n, start, zipf, device=device) for name, r in recipes.items()}
